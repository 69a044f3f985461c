"""The oracle against its pins (no GPU).  See tests/oracle_pins.py."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from tests import oracle_pins as pins


@pytest.fixture(scope="module")
def L():
    return oracle.lib()


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(L, pin):
    bad = pin(L)
    assert not bad, "\n".join(bad[:20])


def test_batch_matches_single(L):
    kb = pins.identity_kb(700)
    okb = oracle.from_synth(kb)
    from synth import hyps
    progs = hyps.small_hyps(kb, 3, 40)
    flat, offs = hyps.batch_arrays(progs)
    for threads in (1, 3):
        counts, sets, errs = oracle.eval_batch(okb, flat, offs, threads=threads, keep_sets=True)
        assert not errs.any()
        for h, p in enumerate(progs):
            r = oracle.eval_program(okb, p)
            assert np.array_equal(sets[h].astype(bool), r)
            assert np.array_equal(counts[h], oracle.score(okb, r))


def test_accuracy_f1():
    acc, f1 = oracle.accuracy_f1(np.array([[3, 1, 1, 3], [0, 0, 4, 4], [0, 0, 0, 0]]))
    assert np.allclose(acc, [0.75, 0.5, 0.0])
    assert np.allclose(f1, [0.75, 0.0, 0.0])


# Planted mistakes: each mutant is a copy of the oracle source with one
# plausible error; at least one pin must reject it.
MUTANTS = {
    "exists_transposed": ("uint32_t a = inverse ? kb->obj[k] : kb->subj[k];   /* the individual being classified */",
                          "uint32_t a = inverse ? kb->subj[k] : kb->obj[k];   /* the individual being classified */"),
    "forall_no_vacuous": ("memset(out, 1, (size_t)kb->n);", "memset(out, 0, (size_t)kb->n);"),
    "atleast_strict": ("out[i] = cnt[i] >= (int64_t)n;", "out[i] = cnt[i] > (int64_t)n;"),
    "atmost_paper_max": ("out[i] = cnt[i] <= (int64_t)n;", "out[i] = cnt[i] > 0 && cnt[i] <= (int64_t)n;"),
    "exactly_as_atleast": ("else out[i] = cnt[i] == (int64_t)n;", "else out[i] = cnt[i] >= (int64_t)n;"),
    "data_strict_ge": ("if (op == O_DGE) out[i] = v[i] >= t;", "if (op == O_DGE) out[i] = v[i] > t;"),
    "data_le_swapped": ("else if (op == O_DLE) out[i] = v[i] <= t;", "else if (op == O_DLE) out[i] = v[i] >= t;"),
    "and_or_swapped": ("(op == O_AND) ? (x[i] & y[i]) : (x[i] | y[i])", "(op == O_AND) ? (x[i] | y[i]) : (x[i] & y[i])"),
    "fn_uses_fp": ("counts[2] = np_ - tp;", "counts[2] = np_ - fp;"),
    "count_ignores_filler": ("if (x[b]) cnt[a] += 1;", "cnt[a] += 1;"),
    "forall_inverse_ignored": ("uint32_t b = inverse ? kb->subj[k] : kb->obj[k];\n        if (!x[b])",
                               "uint32_t b = kb->obj[k];\n        if (!x[b])"),
    "numeric_last_value_wins": ("if (compare(op, kb->num_val[k], t)) out[kb->num_subj[k]] = 1;",
                                "out[kb->num_subj[k]] = (uint8_t)compare(op, kb->num_val[k], t);"),
    "numeric_first_role_only": ("op_numeric_role(kb, op, p - (unsigned)kb->n_props, t, out);",
                                "op_numeric_role(kb, op, 0, t, out);"),
    "numeric_eq_as_ge": ("    return v == t;\n}", "    return v >= t;\n}"),
    "numeric_le_strict": ("if (op == O_DLE) return v <= t;", "if (op == O_DLE) return v < t;"),
    "numeric_ids_rejected": ("(int64_t)a_of(prog[k]) >= (int64_t)kb->n_props + kb->n_num_roles",
                             "(int64_t)a_of(prog[k]) >= (int64_t)kb->n_props"),
    "contain_misses_the_end": ("for (int64_t i = 0; i + lp <= lx; ++i) {", "for (int64_t i = 0; i + lp < lx; ++i) {"),
    "contain_first_char_only": ("while (j < lp && x[i + j] == p[j]) ++j;", "while (j < lp && x[i + j] == p[0]) ++j;"),
    "equal_as_prefix": ("    if (lx != ly) return 0;", "    if (lx < ly) return 0;"),
    "seq_absent_is_first": ("if ((int64_t)b >= kb->n_strings) return;", "if ((int64_t)b >= kb->n_strings) b = 0;"),
    "string_first_role_only": ("for (int64_t k = kb->str_off[s]; k < kb->str_off[s + 1]; ++k) {",
                               "for (int64_t k = kb->str_off[0]; k < kb->str_off[1]; ++k) {"),
    "validate_depth_off_by_one": ("if (depth > ORACLE_MAX_STACK) return OE_OVERFLOW;",
                                  "if (depth >= ORACLE_MAX_STACK) return OE_OVERFLOW;"),
    # the byte model (the per-operation table of algorithmic bytes)
    "bytes_filler_read_only": ("+ 4 * (kb->role_off[a + 1] - kb->role_off[a]) + 2 * B;",
                               "+ 4 * (kb->role_off[a + 1] - kb->role_off[a]) + B;"),
    "bytes_first_role_edges": ("+ 4 * (kb->role_off[a + 1] - kb->role_off[a]) + 2 * B;",
                               "+ 4 * (kb->role_off[1] - kb->role_off[0]) + 2 * B;"),
    "bytes_row_pointers_n": ("return 4 * (n + 1) + 4 * (kb->role_off[a + 1]", "return 4 * n + 4 * (kb->role_off[a + 1]"),
    "bytes_atom_free": ("case O_ATOM: return B;", "case O_ATOM: return 0;"),
    "bytes_unpadded_rows": ("int64_t wp = (w + 3) / 4 * 4;", "int64_t wp = w;"),
    "bytes_score_one_set": ("return 2 * set_bytes(n) + 16;", "return set_bytes(n) + 16;"),
    "bytes_column_plus_one": ("if ((int32_t)a < kb->n_props) return 4 * n;", "if ((int32_t)a < kb->n_props) return 4 * (n + 1);"),
    "bytes_contain_no_bitmap": ("+ 4 * ((kb->n_strings + 31) / 32);", ";"),
    "bytes_not_counts_a_set": ("case O_TOP: case O_BOT: case O_NOT: case O_AND: case O_OR: return 0;",
                               "case O_NOT: return B;\n    case O_TOP: case O_BOT: case O_AND: case O_OR: return 0;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "hedl_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    src = src.replace(old, new, 1)
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "m.c")
        so = os.path.join(d, "m.so")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", so, c, "-lm"])
        M = oracle.load(so)
        failures = []
        for pin in pins.ALL_PINS:
            try:
                failures += pin(M)
            except ValueError as e:          # the mutant rejected a valid program
                failures.append(f"{pin.__name__}: {e}")
            if failures:
                break
        assert failures, f"mutant {name} passed every pin"
