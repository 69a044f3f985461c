"""Pins of the oracle to facts that do not come from the oracle itself.

Each ``pin_*`` function takes a loaded oracle library and returns a list of
failure messages (empty = pinned).  ``tests/test_oracle.py`` runs them on
the real oracle and on deliberately broken copies of it (a planted mistake
must make at least one pin fail).

Sources of truth:
* hand-worked fixtures (tests/golden/*.txt, each with its citations);
* a first-order brute-force evaluator on tiny random KBs (oracle.fo_brute);
* DL identities (De Morgan, double negation, excluded middle, FORALL as
  NOT EXISTS NOT, ATLEAST 1 as EXISTS, ATMOST n as NOT ATLEAST n+1, EXACTLY
  as ATLEAST and ATMOST, ATLEAST 0 as TOP, (r^-)^- = r) -- the oracle computes
  each side by its own code path;
* closed forms on the paper's two role-assertion stress shapes ("single
  subject": one subject holds every assertion; "unique subject": each
  subject one assertion, here a permutation) and on sorted data values;
* the transposed assertion list: EXISTS r^- C on a KB equals EXISTS r C on
  the KB whose role is the (numpy-built) transpose;
* numeric concrete roles (several values per subject, Section III-B,
  Algorithms 9-10): closed forms through per-subject maxima / minima / value
  sets (>= t iff the largest value is >= t, and so on), a hand-worked KB with
  NaN and signed zeros, the single- and unique-subject shapes (the latter
  against a one-value property holding the same values) and the identities
  (>= t) or (<= t) = "has a value", (== t) within both;
* string concrete roles (Algorithms 11-14): a hand-worked KB; closed forms
  through the interned ids (the oracle compares bytes) and Python's own
  substring search over the table; the empty pattern = "has a value"; a
  string's equality restriction within the containment of any of its
  substrings; the brute force over tiny KBs with string roles.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

import oracle
from oracle import fo_brute
from synth import kb as K
from synth import programs as P
from synth.rng import Rng
from tests import golden_io


def tiny_from_fixture(fx):
    okb = oracle.OracleKB.from_parts(
        fx.n,
        np.array([[1 if i in c else 0 for i in range(fx.n)] for c in fx.concept_list()], dtype=np.uint8)
        .reshape(-1, fx.n),
        [(np.array([a for a, _ in es], np.uint32), np.array([b for _, b in es], np.uint32))
         for es in fx.role_list()],
        np.array(fx.prop_rows(), dtype=np.float32).reshape(-1, fx.n),
        np.array([1 if i in fx.pos else 0 for i in range(fx.n)], np.uint8),
        np.array([1 if i in fx.neg else 0 for i in range(fx.n)], np.uint8))
    return okb


def pin_golden(L) -> List[str]:
    bad = []
    for name in golden_io.fixtures():
        fx = golden_io.load(name)
        okb = tiny_from_fixture(fx)
        for q, inst, cnt in fx.queries:
            got = oracle.eval_program(okb, P.compile_text(q), L=L)
            got_set = set(np.nonzero(got)[0].tolist())
            if got_set != inst:
                bad.append(f"{name}: {q}: {sorted(got_set)} != {sorted(inst)}")
            c = tuple(int(x) for x in oracle.score(okb, got, L=L))
            if c != cnt:
                bad.append(f"{name}: {q}: counts {c} != {cnt}")
    return bad


def to_tiny(kb: K.KB) -> fo_brute.TinyKB:
    n = kb.n
    concepts = [set(np.nonzero(K.unpack_bits(kb.concept_bits[c], n))[0].tolist()) for c in range(kb.n_concepts)]
    roles = []
    for r in range(kb.n_roles):
        rp, col = kb.row_ptr[r], kb.col[r]
        roles.append({(a, int(col[k])) for a in range(n) for k in range(int(rp[a]), int(rp[a + 1]))})
    props = [{i: float(v) for i, v in enumerate(kb.prop_vals[p]) if not math.isnan(v)} for p in range(kb.n_props)]
    for q in range(kb.n_num_roles):
        rp, vals = kb.num_row_ptr[q], kb.num_vals[q]
        props.append({i: [float(vals[k]) for k in range(int(rp[i]), int(rp[i + 1]))]
                      for i in range(n) if rp[i + 1] > rp[i]})
    strs = []
    for q in range(kb.n_str_roles):
        rp, ids = kb.str_row_ptr[q], kb.str_ids[q]
        strs.append({i: [kb.strings[int(ids[k])] for k in range(int(rp[i]), int(rp[i + 1]))]
                     for i in range(n) if rp[i + 1] > rp[i]})
    return fo_brute.TinyKB(n, concepts, roles, props, strs, kb.strings, kb.patterns)


def random_program(r: Rng, kb: K.KB, depth: int, role_free: bool = False) -> P.Node:
    """Random tree over every constructor, including TOP, BOT, EXACTLY and DEQ."""
    if depth <= 1 or r.random() < 0.25:
        k = r.randint(0, 9)
        if k == 0:
            return P.Node(P.TOP)
        if k == 1:
            return P.Node(P.BOT)
        if k <= 3 and kb.n_str_roles and r.random() < 0.5:
            q = r.randint(0, kb.n_str_roles - 1)
            if r.random() < 0.5 and kb.n_patterns:
                return P.Node(P.SCONTAINS, q, r.randint(0, kb.n_patterns - 1))
            return P.Node(P.SEQ, q, r.randint(0, len(kb.strings)))    # the last id is not in the table
        if k <= 3 and kb.n_num_roles and r.random() < 0.5:
            q = r.randint(0, kb.n_num_roles - 1)
            vals = kb.num_vals[q]
            t = float(vals[r.randint(0, vals.size - 1)]) if vals.size else 1.0
            return P.Node((P.DGE, P.DLE, P.DEQ)[r.randint(0, 2)], kb.n_props + q, P.f32_bits(t))
        if k <= 3 and kb.n_props:
            p = r.randint(0, kb.n_props - 1)
            vals = kb.prop_vals[p]
            t = float(vals[r.randint(0, kb.n - 1)])
            if math.isnan(t):
                t = float(r.randint(0, 100))
            return P.Node((P.DGE, P.DLE, P.DEQ)[r.randint(0, 2)], p, P.f32_bits(t))
        return P.Node(P.ATOM, r.randint(0, kb.n_concepts - 1))
    k = r.randint(0, 2 if role_free else 8)
    if k == 0:
        return P.Node(P.NOT, kids=[random_program(r, kb, depth - 1, role_free)])
    if k <= 2:
        return P.Node((P.AND, P.OR)[k - 1], kids=[random_program(r, kb, depth - 1, role_free),
                                                  random_program(r, kb, depth - 1, role_free)])
    op = (P.EXISTS, P.FORALL, P.ATLEAST, P.ATMOST, P.EXACTLY, P.EXISTS)[k - 3]
    n = r.randint(0, 4) if op in P.COUNT_OPS else 0
    return P.Node(op, r.randint(0, kb.n_roles - 1), n, r.random() < 0.5, [random_program(r, kb, depth - 1)])


def tiny_kbs():
    base = K.CONFIGS["small"]
    out = []
    for seed, n, deg in ((101, 20, ("poisson", 2.0)), (102, 33, ("poisson", 3.0)), (103, 40, ("poisson", 4.0)),
                         (104, 17, ("zipf", 2.1, 3.0, 16))):
        cfg = base.scaled(n, seed=seed, n_concepts=5, n_roles=3, degree=deg, n_props=2, n_pos=4, n_neg=4)
        out.append(K.generate(cfg))
    for seed, n, nd in ((105, 24, ("poisson", 2.0)), (106, 37, ("poisson", 1.0))):
        cfg = base.scaled(n, seed=seed, n_concepts=4, n_roles=2, degree=("poisson", 2.0), n_props=1, n_pos=4,
                          n_neg=4, n_num_roles=2, num_degree=nd)
        out.append(K.generate(cfg))
    for seed, n in ((107, 29), (108, 41)):
        cfg = base.scaled(n, seed=seed, n_concepts=4, n_roles=2, degree=("poisson", 2.0), n_props=1, n_pos=4,
                          n_neg=4, n_str_roles=2, str_degree=("poisson", 1.5), n_strings=12, str_len=(0, 5),
                          alphabet=3, n_patterns=8)
        out.append(K.generate(cfg))
    return out


def pin_brute_force(L, programs_per_kb: int = 60) -> List[str]:
    bad = []
    for kb in tiny_kbs():
        okb = oracle.from_synth(kb)
        tiny = to_tiny(kb)
        pos = set(kb.pos_idx.tolist())
        neg = set(kb.neg_idx.tolist())
        r = Rng(kb.cfg.seed, 77)
        for i in range(programs_per_kb):
            prog = random_program(r, kb, r.randint(1, 4)).postfix()
            want = fo_brute.evaluate(tiny, prog)
            got = oracle.eval_program(okb, prog, L=L)
            got_set = set(np.nonzero(got)[0].tolist())
            if got_set != want:
                bad.append(f"brute force n={kb.n}: {P.to_text(P.from_postfix(prog))}")
                continue
            if tuple(oracle.score(okb, got, L=L)) != fo_brute.coverage(want, pos, neg):
                bad.append(f"coverage n={kb.n}: {P.to_text(P.from_postfix(prog))}")
    return bad


def _identities(x: str, y: str, r: str, n: int) -> List[tuple]:
    return [
        (f"(not (and {x} {y}))", f"(or (not {x}) (not {y}))"),
        (f"(not (or {x} {y}))", f"(and (not {x}) (not {y}))"),
        (f"(not (not {x}))", x),
        (f"(and {x} (not {x}))", "BOT"),
        (f"(or {x} (not {x}))", "TOP"),
        (f"(all {r} {x})", f"(not (some {r} (not {x})))"),
        (f"(min 1 {r} {x})", f"(some {r} {x})"),
        (f"(max {n} {r} {x})", f"(not (min {n + 1} {r} {x}))"),
        (f"(exactly {n} {r} {x})", f"(and (min {n} {r} {x}) (max {n} {r} {x}))"),
        (f"(min 0 {r} {x})", "TOP"),
        (f"(max 0 {r} {x})", f"(not (some {r} {x}))"),
        (f"(some {r}-- {x})", f"(some {r} {x})"),
    ]


def identity_kb(n: int = 600):
    cfg = K.CONFIGS["small"].scaled(n, seed=31, n_concepts=8, n_roles=3)
    return K.generate(cfg)


def pin_identities(L, kb=None, count: int = 6) -> List[str]:
    kb = kb or identity_kb()
    okb = oracle.from_synth(kb)
    r = Rng(5, 5)
    bad = []
    for i in range(count):
        x = P.to_text(random_program(r, kb, 3))
        y = P.to_text(random_program(r, kb, 2))
        role = f"r{r.randint(0, kb.n_roles - 1)}{'-' if r.random() < 0.5 else ''}"
        n = r.randint(0, 3)
        for lhs, rhs in _identities(x, y, role, n):
            a = oracle.eval_program(okb, P.compile_text(lhs), L=L)
            b = oracle.eval_program(okb, P.compile_text(rhs), L=L)
            if not np.array_equal(a, b):
                bad.append(f"identity {lhs} == {rhs}")
        res = oracle.eval_program(okb, P.compile_text(x), L=L)
        tp, fp, fn, tn = oracle.score(okb, res, L=L)
        if tp + fn != kb.pos_idx.size or fp + tn != kb.neg_idx.size:
            bad.append("TP+FN != |P| or FP+TN != |N|")
        if tp != int(res[kb.pos_idx].sum()) or fp != int(res[kb.neg_idx].sum()):
            bad.append("coverage differs from counting the example indices")
    return bad


def pin_inverse_transpose(L, kb=None) -> List[str]:
    """EXISTS/FORALL/ATLEAST r^- C on a KB equal the forward ops on the transposed KB."""
    kb = kb or identity_kb()
    okb = oracle.from_synth(kb)
    n = kb.n
    edges_t = []
    for r in range(kb.n_roles):
        deg = np.diff(kb.inv_row_ptr[r].astype(np.int64))
        edges_t.append((np.repeat(np.arange(n, dtype=np.uint32), deg), kb.inv_col[r]))
    okb_t = oracle.OracleKB.from_parts(n, okb.member, edges_t, okb.prop, okb.pos, okb.neg)
    bad = []
    r = Rng(6, 6)
    for i in range(8):
        x = P.to_text(random_program(r, kb, 3, role_free=True))
        role = r.randint(0, kb.n_roles - 1)
        for form in ("(some r{}{} X)", "(all r{}{} X)", "(min 2 r{}{} X)", "(max 1 r{}{} X)"):
            a = oracle.eval_program(okb, P.compile_text(form.format(role, "-").replace("X", x)), L=L)
            b = oracle.eval_program(okb_t, P.compile_text(form.format(role, "").replace("X", x)), L=L)
            if not np.array_equal(a, b):
                bad.append(f"inverse vs transpose {form}")
    return bad


def pin_closed_forms(L) -> List[str]:
    bad = []
    base = K.CONFIGS["small"]
    # unique subject: role r is a permutation pi (a -> pi(a))
    kb = K.generate(base.scaled(257, seed=41, n_concepts=4, n_roles=1, degree=("unique",)))
    okb = oracle.from_synth(kb)
    pi = kb.col[0].astype(np.int64)
    for c in range(kb.n_concepts):
        C = K.unpack_bits(kb.concept_bits[c], kb.n)
        pre = C[pi]                                   # {a : pi(a) in C}
        img = np.zeros(kb.n, bool)
        img[pi[C]] = True                             # {pi(a) : a in C}
        checks = [(f"(some r0 A{c})", pre), (f"(all r0 A{c})", pre), (f"(some r0- A{c})", img),
                  (f"(min 2 r0 A{c})", np.zeros(kb.n, bool)), (f"(max 0 r0 A{c})", ~pre),
                  (f"(exactly 1 r0- A{c})", img)]
        for q, want in checks:
            if not np.array_equal(oracle.eval_program(okb, P.compile_text(q), L=L), want):
                bad.append(f"unique subject: {q}")
    # single subject: subject s holds every assertion, to targets T
    kb = K.generate(base.scaled(300, seed=42, n_concepts=4, n_roles=1, degree=("single", 120)))
    okb = oracle.from_synth(kb)
    s = int(np.nonzero(np.diff(kb.row_ptr[0].astype(np.int64)))[0][0])
    T = np.zeros(kb.n, bool)
    T[kb.col[0]] = True
    for c in range(kb.n_concepts):
        C = K.unpack_bits(kb.concept_bits[c], kb.n)
        k = int((C & T).sum())
        only_s = np.zeros(kb.n, bool)
        only_s[s] = True
        none = np.zeros(kb.n, bool)
        allx = np.ones(kb.n, bool)
        checks = [(f"(some r0 A{c})", only_s if k > 0 else none),
                  (f"(min {k} r0 A{c})", only_s if k > 0 else allx),
                  (f"(min {k + 1} r0 A{c})", none),
                  (f"(exactly {k} r0 A{c})", only_s if k > 0 else allx),
                  (f"(all r0 A{c})", allx if not (T & ~C).any() else ~only_s),
                  (f"(some r0- A{c})", T if C[s] else none),
                  (f"(max {max(k - 1, 0)} r0 A{c})", ~only_s if k > 0 else allx)]
        for q, want in checks:
            if not np.array_equal(oracle.eval_program(okb, P.compile_text(q), L=L), want):
                bad.append(f"single subject: {q}")
    # data ranges: counts from sorted present values (searchsorted)
    kb = K.generate(base.scaled(5000, seed=43, n_concepts=1, n_roles=1))
    okb = oracle.from_synth(kb)
    for p in range(kb.n_props):
        v = kb.prop_vals[p]
        pres = np.sort(v[~np.isnan(v)])
        for t in (float(pres[0]), float(pres[len(pres) // 3]), float(pres[-1]), -0.0, 0.0, 50.0,
                  math.inf, -math.inf):
            t32 = np.float32(t)
            ge = len(pres) - int(np.searchsorted(pres, t32, side="left"))
            le = int(np.searchsorted(pres, t32, side="right"))
            eq = le - int(np.searchsorted(pres, t32, side="left"))
            for op, want in ((P.DGE, ge), (P.DLE, le), (P.DEQ, eq)):
                got = int(oracle.eval_program(okb, [P.insn(op, 0, p, P.f32_bits(t))], L=L).sum())
                if got != want:
                    bad.append(f"data closed form op={op} t={t}: {got} != {want}")
    return bad


def _per_subject(kb, q):
    """(has a value, largest value, smallest value, subject of each value) of numeric role q."""
    rp = kb.num_row_ptr[q].astype(np.int64)
    vals = kb.num_vals[q].astype(np.float32)
    subj = np.repeat(np.arange(kb.n), np.diff(rp))
    present = ~np.isnan(vals)
    has = np.zeros(kb.n, bool)
    has[subj[present]] = True
    mx = np.full(kb.n, -np.inf, np.float32)
    np.maximum.at(mx, subj[present], vals[present])
    mn = np.full(kb.n, np.inf, np.float32)
    np.minimum.at(mn, subj[present], vals[present])
    return has, mx, mn, subj, vals


def pin_numeric_roles(L) -> List[str]:
    bad = []
    base = K.CONFIGS["small"]
    ev = lambda okb, op, p, t: oracle.eval_program(okb, [P.insn(op, 0, p, P.f32_bits(t))], L=L)
    # closed forms: some value >= t iff the largest is; <= t iff the smallest is; == t iff t is among them
    for seed, n, nd in ((111, 300, ("poisson", 2.5)), (112, 97, ("single", 40)), (113, 200, ("unique",))):
        kb = K.generate(base.scaled(n, seed=seed, n_concepts=2, n_roles=1, degree=("poisson", 2.0), n_props=1,
                                    n_pos=10, n_neg=10, n_num_roles=3, num_degree=nd))
        okb = oracle.from_synth(kb)
        for q in range(kb.n_num_roles):
            has, mx, mn, subj, vals = _per_subject(kb, q)
            srt = np.sort(vals)
            for t in (float(srt[0]), float(srt[len(srt) // 2]), float(srt[-1]), float(np.nextafter(srt[-1], 2e3)),
                      -0.0, 0.0, 500.0, math.inf, -math.inf):
                t32 = np.float32(t)
                eq = np.zeros(kb.n, bool)
                eq[subj[vals == t32]] = True
                for op, want in ((P.DGE, has & (mx >= t32)), (P.DLE, has & (mn <= t32)), (P.DEQ, eq)):
                    if not np.array_equal(ev(okb, op, kb.n_props + q, t), want):
                        bad.append(f"numeric closed form {nd[0]} q={q} op={op} t={t}")
                ge, le, eqs = (ev(okb, op, kb.n_props + q, t) for op in (P.DGE, P.DLE, P.DEQ))
                if not np.array_equal(ge | le, has) or (eqs & ~(ge & le)).any():
                    bad.append(f"numeric identities {nd[0]} q={q} t={t}")
            if nd[0] == "single":
                r = ev(okb, P.DGE, kb.n_props + q, float(srt[0]))
                if int(r.sum()) != 1 or not r[subj[0]]:
                    bad.append(f"single subject q={q}: {np.nonzero(r)[0].tolist()}")
            if nd[0] == "unique":
                # one value per subject: the same as a one-value property holding those values
                col = np.full(kb.n, np.nan, np.float32)
                col[subj] = vals
                dense = oracle.OracleKB.from_parts(kb.n, np.zeros((0, kb.n), np.uint8), [], col[None, :],
                                                   okb.pos, okb.neg)
                for t in (float(srt[3]), float(srt[-5]), 0.0):
                    for op in (P.DGE, P.DLE, P.DEQ):
                        if not np.array_equal(ev(okb, op, kb.n_props + q, t), ev(dense, op, 0, t)):
                            bad.append(f"unique subject q={q} op={op} t={t}")
    # an existential restriction ignores how often a value is asserted: the KB with every numeric
    # assertion doubled (in another order) gives the same sets
    kb = K.generate(base.scaled(250, seed=114, n_concepts=2, n_roles=1, degree=("poisson", 2.0), n_props=1,
                                n_pos=10, n_neg=10, n_num_roles=2, num_degree=("poisson", 2.0)))
    okb = oracle.from_synth(kb)
    pairs = []
    for q in range(kb.n_num_roles):
        _, _, _, subj, vals = _per_subject(kb, q)
        pairs.append((np.concatenate([subj[::-1], subj]), np.concatenate([vals[::-1], vals])))
    dup = oracle.OracleKB.from_parts(kb.n, okb.member, [], okb.prop, okb.pos, okb.neg, pairs)
    for q in range(kb.n_num_roles):
        for t in (float(np.median(kb.num_vals[q])), 0.0):
            for op in (P.DGE, P.DLE, P.DEQ):
                if not np.array_equal(ev(okb, op, kb.n_props + q, t), ev(dup, op, kb.n_props + q, t)):
                    bad.append(f"numeric duplicates q={q} op={op} t={t}")
    # hand-worked: individual 0 holds {1.5, NaN}, 2 holds {-0.0}, 3 holds {NaN},
    # 4 holds {7, 2, 9}, 5 holds {+0.0}; 1 holds nothing (a missing value)
    nan = float("nan")
    a = [(4, 7.0), (0, 1.5), (2, -0.0), (4, 2.0), (3, nan), (0, nan), (4, 9.0), (5, 0.0)]
    okb = oracle.OracleKB.from_parts(6, np.zeros((0, 6), np.uint8), [], np.full((1, 6), np.nan, np.float32),
                                     np.zeros(6, np.uint8), np.zeros(6, np.uint8),
                                     [(np.array([s for s, _ in a]), np.array([v for _, v in a], np.float32))])
    for op, t, want in ((P.DGE, 2.0, {4}), (P.DLE, 1.5, {0, 2, 5}), (P.DEQ, 0.0, {2, 5}), (P.DEQ, -0.0, {2, 5}),
                        (P.DEQ, 2.0, {4}), (P.DEQ, nan, set()), (P.DGE, nan, set()), (P.DGE, -math.inf, {0, 2, 4, 5}),
                        (P.DLE, math.inf, {0, 2, 4, 5}), (P.DGE, 9.5, set()), (P.DLE, -1.0, set())):
        got = set(np.nonzero(ev(okb, op, 1, t))[0].tolist())
        if got != want:
            bad.append(f"hand-worked numeric role op={op} t={t}: {sorted(got)} != {sorted(want)}")
    return bad


def pin_string_roles(L) -> List[str]:
    bad = []
    ins = lambda op, s_, b: [P.insn(op, 0, s_, b)]
    sets = lambda okb, op, s_, b: set(np.nonzero(oracle.eval_program(okb, ins(op, s_, b), L=L))[0].tolist())
    # hand-worked: role 0 asserts 0:{catalog, dog} 1:{cat} 2:{""} 3:{at, dog} 5:{catalog}; role 1 asserts 4:{dog}
    strings = [b"cat", b"catalog", b"dog", b"", b"at"]
    patterns = [b"", b"cat", b"og", b"atalogue", b"t", b"a"]
    r0 = [(5, b"catalog"), (0, b"dog"), (1, b"cat"), (2, b""), (3, b"at"), (0, b"catalog"), (3, b"dog")]
    z = np.zeros(6, np.uint8)
    okb = oracle.OracleKB.from_parts(6, np.zeros((0, 6), np.uint8), [], np.zeros((0, 6), np.float32), z, z,
                                     str_roles=[(np.array([a for a, _ in r0]), [v for _, v in r0]),
                                                (np.array([4]), [b"dog"])],
                                     strings=strings, patterns=patterns)
    cases = [(P.SEQ, 0, 0, {1}), (P.SEQ, 0, 1, {0, 5}), (P.SEQ, 0, 2, {0, 3}), (P.SEQ, 0, 3, {2}),
             (P.SEQ, 0, 4, {3}), (P.SEQ, 0, 5, set()), (P.SEQ, 0, 0xFFFFFFFF, set()), (P.SEQ, 1, 2, {4}),
             (P.SEQ, 1, 0, set()), (P.SCONTAINS, 0, 0, {0, 1, 2, 3, 5}), (P.SCONTAINS, 0, 1, {0, 1, 5}),
             (P.SCONTAINS, 0, 2, {0, 3, 5}), (P.SCONTAINS, 0, 3, set()), (P.SCONTAINS, 0, 4, {0, 1, 3, 5}),
             (P.SCONTAINS, 0, 5, {0, 1, 3, 5}), (P.SCONTAINS, 1, 2, {4}), (P.SCONTAINS, 1, 1, set())]
    for op, s_, b, want in cases:
        got = sets(okb, op, s_, b)
        if got != want:
            bad.append(f"hand-worked string role op={op} s={s_} b={b}: {sorted(got)} != {sorted(want)}")
    # generated KBs: closed forms through the interned ids and Python's substring search
    base = K.CONFIGS["small"]
    for seed, n, sd in ((121, 400, ("poisson", 2.0)), (122, 150, ("single", 60)), (123, 300, ("unique",))):
        kb = K.generate(base.scaled(n, seed=seed, n_concepts=2, n_roles=1, degree=("poisson", 2.0), n_props=1,
                                    n_pos=10, n_neg=10, n_str_roles=2, str_degree=sd, n_strings=40,
                                    str_len=(1, 7), alphabet=4, n_patterns=10))
        okb = oracle.from_synth(kb)
        contains = [[p_ in x for x in kb.strings] for p_ in kb.patterns]
        for q in range(kb.n_str_roles):
            ids = kb.str_ids[q].astype(np.int64)
            subj = np.repeat(np.arange(kb.n), np.diff(kb.str_row_ptr[q].astype(np.int64)))
            has = set(subj.tolist())
            seq = {}
            for b in list(range(len(kb.strings))) + [len(kb.strings), 0xFFFFFFFF]:
                want = set(subj[ids == b].tolist())
                seq[b] = sets(okb, P.SEQ, q, b)
                if seq[b] != want:
                    bad.append(f"string closed form SEQ {sd[0]} q={q} b={b}")
            for k in range(len(kb.patterns)):
                hit = np.array(contains[k], bool)
                want = set(subj[hit[ids]].tolist()) if ids.size else set()
                got = sets(okb, P.SCONTAINS, q, k)
                if got != want:
                    bad.append(f"string closed form SCONTAINS {sd[0]} q={q} k={k}")
                if kb.patterns[k] == b"" and got != has:
                    bad.append(f"empty pattern {sd[0]} q={q}")
                for b, x in enumerate(kb.strings):      # equal to x implies containing any substring of x
                    if kb.patterns[k] in x and not seq[b] <= got:
                        bad.append(f"SEQ within SCONTAINS {sd[0]} q={q} b={b} k={k}")
                        break
    return bad


def pin_validation(L) -> List[str]:
    fx = golden_io.load("family.txt")
    okb = tiny_from_fixture(fx)
    A = lambda c: P.insn(P.ATOM, 0, c)
    cases = [
        ([], -6),
        ([P.insn(0)], -1),
        ([P.insn(17)], -1),
        ([P.insn(255)], -1),
        ([A(4)], -2),
        ([A(0), P.insn(P.EXISTS, 0, 2)], -2),
        ([P.insn(P.DGE, 0, 1, 0)], -2),
        ([A(0), P.insn(P.AND)], -3),
        ([P.insn(P.NOT)], -3),
        ([A(0), A(1)], -5),
        ([A(0)] * 65 + [P.insn(P.AND)] * 64, -4),
        ([A(0)] * 64 + [P.insn(P.AND)] * 63, 0),
    ]
    bad = []
    for prog, want in cases:
        got = oracle.validate(okb, np.array(prog, dtype=np.uint64), L=L)
        if got != want:
            bad.append(f"validate {prog[:3]}...: {got} != {want}")
    # property ids: n_props one-value properties, then the numeric concrete roles
    nkb = oracle.OracleKB.from_parts(3, np.zeros((0, 3), np.uint8), [], np.zeros((2, 3), np.float32),
                                     np.zeros(3, np.uint8), np.zeros(3, np.uint8),
                                     [(np.array([0]), np.array([1.0]))] * 2)
    for p, want in ((1, 0), (2, 0), (3, 0), (4, -2)):
        got = oracle.validate(nkb, np.array([P.insn(P.DGE, 0, p, 0)], dtype=np.uint64), L=L)
        if got != want:
            bad.append(f"validate property id {p}: {got} != {want}")
    # string roles: role ids below n_str_roles; pattern ids below n_patterns; any string id
    z = np.zeros(3, np.uint8)
    skb = oracle.OracleKB.from_parts(3, np.zeros((0, 3), np.uint8), [], np.zeros((0, 3), np.float32), z, z,
                                     str_roles=[(np.array([0]), [b"x"])] * 2, strings=[b"x"], patterns=[b"", b"x"])
    for op, a, b, want in ((P.SEQ, 1, 0, 0), (P.SEQ, 2, 0, -2), (P.SEQ, 0, 0xFFFFFFFF, 0), (P.SCONTAINS, 1, 1, 0),
                           (P.SCONTAINS, 1, 2, -2), (P.SCONTAINS, 2, 0, -2)):
        got = oracle.validate(skb, np.array([P.insn(op, 0, a, b)], dtype=np.uint64), L=L)
        if got != want:
            bad.append(f"validate string op={op} a={a} b={b}: {got} != {want}")
    return bad


def _bytes_kb(n: int):
    """A hand-built KB for the byte model: 2 concepts, role 0 with 7 assertions and role 1 with 3,
    one one-value property, numeric role 0 with 5 values, string role 0 with 4 values, a table of
    40 strings and 2 patterns."""
    z = np.zeros(n, np.uint8)
    r0 = (np.array([0, 0, 1, 2, 3, 5, 9]) % n, np.array([1, 2, 0, 4, 4, 6, 8]) % n)
    r1 = (np.array([0, 2, 7]) % n, np.array([3, 3, 7]) % n)
    if n < 10:   # keep the pairs a set on tiny KBs
        r0 = (np.array([0, 0, 1, 2, 3, 4, 5])[:7] % n, np.array([1, 2, 0, 4, 4, 6, 8])[:7] % n)
        keys = sorted(set(zip(r0[0].tolist(), r0[1].tolist())))
        r0 = (np.array([a for a, _ in keys]), np.array([b for _, b in keys]))
        keys = sorted(set(zip(r1[0].tolist(), r1[1].tolist())))
        r1 = (np.array([a for a, _ in keys]), np.array([b for _, b in keys]))
    strings = [bytes([97 + i % 26, 98 + i // 26]) for i in range(40)]
    return oracle.OracleKB.from_parts(
        n, np.zeros((2, n), np.uint8), [r0, r1], np.zeros((1, n), np.float32), z, z,
        num_roles=[(np.arange(5) % n, np.arange(5, dtype=np.float32))],
        str_roles=[(np.arange(4) % n, [b"ab", b"cb", b"xx", b""])], strings=strings, patterns=[b"a", b"b"])


def pin_byte_model(L) -> List[str]:
    """The algorithmic-byte model of the plain method (per operation, no sharing credit), counted
    by the oracle while it evaluates.  Pinned to values worked by hand from the per-operation table
    (a set is B = 4 Wp bytes, Wp = ceil(n / 32) rounded up to a multiple of 4; a role restriction
    reads 4(n+1) row-pointer bytes and 4 bytes per assertion of its role and writes and reads its
    filler, 2B; a one-value data restriction reads 4n; a concrete-role restriction 4(n+1) + 4M,
    SCONTAINS also its bitmap row of 4 ceil(S / 32); the score 2B + 16), and to its invariants:
    Boolean operators cost nothing beyond their operands, an inverse costs what its forward role
    does, and B steps at multiples of 128 individuals."""
    bad = []
    t = P.f32_bits(1.0)
    # n = 100: W = 4, Wp = 4, B = 16; score 48; role 0: 404 + 28 + 32 = 464; role 1: 404 + 12 + 32 = 448
    okb = _bytes_kb(100)
    hand = [("A0", 64), ("(some r0 A0)", 528), ("(some r0- A0)", 528), ("(all r1 A1)", 512),
            ("(not (and A0 A1))", 80), ("(or A0 (not A0))", 80), ("TOP", 48), ("(not BOT)", 48),
            ("(min 2 r0 (some r1 A1))", 976), ("(max 1 r1- (exactly 3 r0 A1))", 976)]
    for text, want in hand:
        got = oracle.model_bytes(okb, P.compile_text(text), L=L)
        if got != want:
            bad.append(f"byte model n=100 {text}: {got} != {want}")
    leaves = [([P.insn(P.DGE, 0, 0, t)], 448),                 # 4n + 48
              ([P.insn(P.DLE, 0, 1, t)], 472),                 # numeric role: 404 + 20 + 48
              ([P.insn(P.SEQ, 0, 0, 1)], 468),                 # 404 + 16 + 48
              ([P.insn(P.SCONTAINS, 0, 0, 1)], 476)]           # 404 + 16 + 4 * 2 + 48
    for prog, want in leaves:
        got = oracle.model_bytes(okb, prog, L=L)
        if got != want:
            bad.append(f"byte model n=100 leaf {P.fields(prog[0])}: {got} != {want}")
    # B = 16 up to 128 individuals, 32 from 129 (W = 5 words pad to 8): an atom costs B, its score 2B + 16
    for n, want in ((1, 64), (128, 64), (129, 112), (513, 256)):
        got = oracle.model_bytes(_bytes_kb(n), P.compile_text("A0"), L=L)
        if got != want:
            bad.append(f"byte model n={n} A0: {got} != {want}")
    # invariants on a generated KB: Boolean operators add nothing, inverse = forward, the role
    # term differs between roles by 4 bytes per assertion
    kb = K.generate(K.CONFIGS["small"].scaled(3000, seed=47, n_concepts=6, n_roles=3))
    okb = oracle.from_synth(kb)
    mb = lambda x: oracle.model_bytes(okb, P.compile_text(x), L=L)
    score = mb("TOP")
    for x, y in (("A1", "(some r0 A2)"), ("(min 2 r1 A3)", "(all r2- (or A0 A4))")):
        if mb(f"(and {x} {y})") != mb(x) + mb(y) - score or mb(f"(or {x} (not {y}))") != mb(x) + mb(y) - score:
            bad.append(f"byte model: Boolean operators over {x}, {y} are not free")
    for r in range(kb.n_roles):
        if mb(f"(some r{r}- A0)") != mb(f"(some r{r} A0)"):
            bad.append(f"byte model: inverse of r{r} differs")
    if mb("(some r1 A0)") - mb("(some r0 A0)") != 4 * (kb.n_edges(1) - kb.n_edges(0)):
        bad.append("byte model: role terms do not differ by 4 bytes per assertion")
    return bad


ALL_PINS = (pin_golden, pin_brute_force, pin_identities, pin_inverse_transpose, pin_closed_forms,
            pin_numeric_roles, pin_string_roles, pin_validation, pin_byte_model)
