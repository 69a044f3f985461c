"""Pins of the search oracle (oracle/search.py) that do not use it to check
itself: canonical forms against commuted and nested rewrites, and a one-step
beam over an enumerated candidate space against the first-order brute-force
evaluator's scores sorted by the total order."""
import itertools

import numpy as np

import oracle
from oracle import fo_brute
from oracle import search as OS
from synth import kb as K, programs as P
from tests import oracle_pins as pins


def _c(text):
    return P.compile_text(text)


def test_canonical_form_of_commuted_programs():
    a = OS.canonical(_c("(and A1 (or (some r0 A2) A0))"))
    b = OS.canonical(_c("(and (or A0 (some r0 A2)) A1)"))
    assert a == b
    # idempotent: the canonical program is its own canonical form
    assert OS.canonical(np.frombuffer(a, np.uint64)) == a
    # non-commutative structure stays: a restriction's filler is not swapped with anything
    assert OS.canonical(_c("(some r0 (and A1 A2))")) != OS.canonical(_c("(and (some r0 A1) A2)"))
    # NOT keeps its operand; different operands give different forms
    assert OS.canonical(_c("(not (and A1 A2))")) == OS.canonical(_c("(not (and A2 A1))"))
    assert OS.canonical(_c("(and A1 (not A2))")) != OS.canonical(_c("(and (not A1) A2)"))
    # operand order is by instruction bytes: the form of (and X Y) starts with the smaller operand
    x, y = _c("A3"), _c("(some r1 A0)")
    first = min(x.tobytes(), y.tobytes())
    assert OS.canonical(_c("(and (some r1 A0) A3)")).startswith(first)


def _space(kb):
    """Every program of a small space: atoms, their negations, their pairwise conjunctions,
    and one existential restriction per (role, direction, atom)."""
    out = []
    for c in range(kb.n_concepts):
        out += [f"A{c}", f"(not A{c})"]
    for c, d in itertools.combinations(range(kb.n_concepts), 2):
        out.append(f"(and A{c} A{d})")
    for r in range(kb.n_roles):
        for inv in ("", "-"):
            for c in range(kb.n_concepts):
                out.append(f"(some r{r}{inv} A{c})")
    return [_c(t) for t in out]


def test_one_step_beam_is_the_top_of_an_enumerated_space():
    kb = pins.tiny_kbs()[1]
    tiny = pins.to_tiny(kb)
    pos = set(np.nonzero(K.unpack_bits(kb.pos_bits, kb.n))[0].tolist())
    neg = set(np.nonzero(K.unpack_bits(kb.neg_bits, kb.n))[0].tolist())
    space = _space(kb)
    start = [_c("TOP")]
    # scores by first-order brute force, an evaluator independent of the C oracle
    def brute(prog):
        tp, fp, fn, tn = fo_brute.coverage(fo_brute.evaluate(tiny, prog), pos, neg)
        tot = tp + fp + fn + tn
        den = 2 * tp + fp + fn
        return (tp + tn) / tot, (2 * tp / den if den else 0.0), (tp, fp, fn, tn)
    cands = [start[0]] + space
    scored = [brute(p) for p in cands]
    width = 12

    def refine(beam, step, count):
        assert step == 1
        return list(space)

    beam = OS.exhaustive(oracle.from_synth(kb), refine, start, 1, width, len(space))
    assert len(beam) == width
    # the beam's accuracies are the top `width` accuracies of start + space, best first
    want_acc = sorted((s[0] for s in scored), reverse=True)[:width]
    got = [brute(np.frombuffer(b, np.uint64)) for b, _ in beam]
    assert [g[0] for g in got] == want_acc
    # counts reported by the search are the brute-force counts
    assert [c for _, c in beam] == [g[2] for g in got]
    # ties in accuracy are broken by F1 (desc), then program length (asc)
    for (a, b) in zip(got, got[1:]):
        assert (a[0], a[1]) >= (b[0], b[1])
    keys = [(-g[0], -g[1], len(b) // 8) for g, (b, _) in zip(got, beam)]
    assert keys == sorted(keys)


def test_commuted_duplicates_count_once():
    kb = pins.tiny_kbs()[0]
    start = [_c("A0")]

    def refine(beam, step, count):
        return [_c("(and A1 A2)"), _c("(and A2 A1)"), _c("(or A3 A4)"), _c("(or A4 A3)"), _c("A0")]

    beam = OS.exhaustive(oracle.from_synth(kb), refine, start, 1, 10, 5)
    forms = [b for b, _ in beam]
    assert len(forms) == len(set(forms)) == 3
