/*
 * hedl_oracle.c -- plain CPU set-semantics evaluator for ALCQI(D) hypotheses.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the oracle that the GPU path is checked
 * against.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never does.  It shares no code,
 * header, table or constant with the GPU library.
 *
 * Representation (the paper's own, Section III-A): one byte per membership
 * (1 = member), a concept's memberships of all individuals contiguous (the
 * transposed concepts matrix); role assertions as a 2-column (subject, object)
 * matrix grouped per role through an offset table; a numeric data property as
 * one float per individual, NaN where the individual has no value; a numeric
 * concrete role (Section III-B: a subject may assert several values) as a
 * 2-column (subject, value) matrix grouped per role through its own offset
 * table.  Property ids below n_props name the one-value properties, ids
 * n_props + q the numeric concrete role q.  A string concrete role is a
 * 2-column (subject, string value) matrix grouped per role, each assertion
 * holding its own bytes; a string table (the strings SEQ names by index) and
 * a pattern list (the substrings SCONTAINS names by index) complete it.
 *
 * Semantics (closed world, Section III-A: anything not asserted is false):
 *   ATOM c         members of c
 *   TOP / BOT      every individual / none
 *   NOT X          complement of X within the n individuals
 *   AND / OR       intersection / union                       (Algorithms 1-2)
 *   EXISTS r X     { a : some assertion r(a,b) with b in X }   (Algorithms 3-4)
 *   FORALL r X     { a : every assertion r(a,b) has b in X };
 *                  an individual with no r-assertion belongs   (Algorithms 5-6)
 *   ATLEAST r n X  { a : #{b : r(a,b), b in X} >= n }
 *   ATMOST  r n X  { a : #{b : r(a,b), b in X} <= n }  (count 0 included)
 *   EXACTLY r n X  { a : #{b : r(a,b), b in X} == n }          (Algorithms 7-8)
 *   inverse r^-    the same with subject and object swapped    (Section III-B)
 *   DGE p t        { a : a has a value v of p and v >= t }
 *   DLE p t        { a : a has a value v of p and v <= t }
 *   DEQ p t        { a : a has a value v of p and v == t }     (Algorithms 9-10)
 *                  (float32 compares; a missing value satisfies nothing; on a
 *                  numeric concrete role "a value" ranges over every
 *                  assertion of the subject: an existential restriction)
 *   SEQ s v        { a : a has a value of string role s equal, byte for
 *                  byte, to table string v }; empty when v is not in the
 *                  table                                       (Algorithms 11-12)
 *   SCONTAINS s k  { a : a has a value of string role s that contains
 *                  pattern k as a substring; the empty pattern is contained
 *                  in every string }                           (Algorithms 13-14)
 * Coverage (Algorithm 15): TP = |R & P|, FP = |R & N|; FN = |P| - TP and
 * TN = |N| - FP complete the confusion matrix.
 *
 * FORALL is computed directly from its definition, not as NOT EXISTS NOT, so
 * that the identity between the two is a real check.  Role assertions are a
 * set (unique-name assumption, Section III-A): the caller supplies each
 * (subject, object) pair at most once, so a count of assertions is a count of
 * distinct successors.
 *
 * Program format: postfix, one uint64 per instruction,
 *   op = bits 0..7, flags = bits 8..15 (bit 0 = inverse role),
 *   a = bits 16..31 (concept / role / property id), b = bits 32..63 (n, or the
 *   float32 bits of a threshold).  Op codes are listed below.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_ATOM 1
#define O_TOP 2
#define O_BOT 3
#define O_NOT 4
#define O_AND 5
#define O_OR 6
#define O_EXISTS 7
#define O_FORALL 8
#define O_ATLEAST 9
#define O_ATMOST 10
#define O_EXACTLY 11
#define O_DGE 12
#define O_DLE 13
#define O_DEQ 14
#define O_SEQ 15
#define O_SCONTAINS 16

#define ORACLE_MAX_STACK 64

/* error codes */
#define OE_OK 0
#define OE_BAD_OP (-1)
#define OE_BAD_ID (-2)
#define OE_UNDERFLOW (-3)
#define OE_OVERFLOW (-4)
#define OE_NOT_ONE (-5)
#define OE_EMPTY (-6)
#define OE_NOMEM (-7)

typedef struct {
    int64_t n;                       /* number of individuals */
    int32_t n_concepts;
    const uint8_t *concept_member;   /* [n_concepts][n] */
    int32_t n_roles;
    const int64_t *role_off;         /* [n_roles + 1] */
    const uint32_t *subj;            /* [total assertions] */
    const uint32_t *obj;
    int32_t n_props;
    const float *prop;               /* [n_props][n] */
    int32_t n_num_roles;             /* numeric concrete roles (property ids n_props + q) */
    const int64_t *num_off;          /* [n_num_roles + 1] */
    const uint32_t *num_subj;        /* [total numeric assertions] */
    const float *num_val;
    int32_t n_str_roles;             /* string concrete roles (ids of SEQ / SCONTAINS) */
    const int64_t *str_off;          /* [n_str_roles + 1]: the assertions of each role */
    const uint32_t *str_subj;        /* [total string assertions] */
    const int64_t *str_val_off;      /* [total string assertions + 1]: each value's bytes */
    const uint8_t *str_val;
    int64_t n_strings;               /* the table SEQ's second field indexes */
    const int64_t *tbl_off;          /* [n_strings + 1] */
    const uint8_t *tbl;
    int64_t n_patterns;              /* the patterns SCONTAINS's second field indexes */
    const int64_t *pat_off;          /* [n_patterns + 1] */
    const uint8_t *pat;
} oracle_kb;

static unsigned op_of(uint64_t w) { return (unsigned)(w & 0xFF); }
static unsigned flags_of(uint64_t w) { return (unsigned)((w >> 8) & 0xFF); }
static unsigned a_of(uint64_t w) { return (unsigned)((w >> 16) & 0xFFFF); }
static uint32_t b_of(uint64_t w) { return (uint32_t)(w >> 32); }

static float as_float(uint32_t bits) {
    float f;
    memcpy(&f, &bits, sizeof f);
    return f;
}

/* Stack effect of each op: how many operands it pops (leaves pop 0). */
static int arity(unsigned op) {
    switch (op) {
    case O_ATOM: case O_TOP: case O_BOT: case O_DGE: case O_DLE: case O_DEQ: case O_SEQ: case O_SCONTAINS:
        return 0;
    case O_NOT: case O_EXISTS: case O_FORALL: case O_ATLEAST: case O_ATMOST: case O_EXACTLY: return 1;
    case O_AND: case O_OR: return 2;
    default: return -1;
    }
}

/* Check a program without evaluating it; returns OE_OK or the first error. */
int oracle_validate(const oracle_kb *kb, const uint64_t *prog, int64_t len) {
    int depth = 0;
    if (len <= 0) return OE_EMPTY;
    for (int64_t k = 0; k < len; ++k) {
        unsigned op = op_of(prog[k]);
        int ar = arity(op);
        if (ar < 0) return OE_BAD_OP;
        if (op == O_ATOM && (int32_t)a_of(prog[k]) >= kb->n_concepts) return OE_BAD_ID;
        if (ar == 1 && op != O_NOT && (int32_t)a_of(prog[k]) >= kb->n_roles) return OE_BAD_ID;
        if ((op == O_DGE || op == O_DLE || op == O_DEQ) &&
            (int64_t)a_of(prog[k]) >= (int64_t)kb->n_props + kb->n_num_roles)
            return OE_BAD_ID;
        if ((op == O_SEQ || op == O_SCONTAINS) && (int32_t)a_of(prog[k]) >= kb->n_str_roles) return OE_BAD_ID;
        if (op == O_SCONTAINS && (int64_t)b_of(prog[k]) >= kb->n_patterns) return OE_BAD_ID;
        if (depth < ar) return OE_UNDERFLOW;
        depth = depth - ar + 1;
        if (depth > ORACLE_MAX_STACK) return OE_OVERFLOW;
    }
    return depth == 1 ? OE_OK : OE_NOT_ONE;
}

/* ---------------------------------------------------------------- operators */

static void op_exists(const oracle_kb *kb, unsigned r, int inverse, const uint8_t *x, uint8_t *out) {
    memset(out, 0, (size_t)kb->n);
    for (int64_t k = kb->role_off[r]; k < kb->role_off[r + 1]; ++k) {
        uint32_t a = inverse ? kb->obj[k] : kb->subj[k];   /* the individual being classified */
        uint32_t b = inverse ? kb->subj[k] : kb->obj[k];   /* its successor */
        if (x[b]) out[a] = 1;
    }
}

static void op_forall(const oracle_kb *kb, unsigned r, int inverse, const uint8_t *x, uint8_t *out) {
    memset(out, 1, (size_t)kb->n);
    for (int64_t k = kb->role_off[r]; k < kb->role_off[r + 1]; ++k) {
        uint32_t a = inverse ? kb->obj[k] : kb->subj[k];
        uint32_t b = inverse ? kb->subj[k] : kb->obj[k];
        if (!x[b]) out[a] = 0;
    }
}

static void op_count(const oracle_kb *kb, unsigned op, unsigned r, int inverse, uint32_t n,
                     const uint8_t *x, uint8_t *out, int64_t *cnt) {
    memset(cnt, 0, (size_t)kb->n * sizeof(int64_t));
    for (int64_t k = kb->role_off[r]; k < kb->role_off[r + 1]; ++k) {
        uint32_t a = inverse ? kb->obj[k] : kb->subj[k];
        uint32_t b = inverse ? kb->subj[k] : kb->obj[k];
        if (x[b]) cnt[a] += 1;
    }
    for (int64_t i = 0; i < kb->n; ++i) {
        if (op == O_ATLEAST) out[i] = cnt[i] >= (int64_t)n;
        else if (op == O_ATMOST) out[i] = cnt[i] <= (int64_t)n;
        else out[i] = cnt[i] == (int64_t)n;
    }
}

static int compare(unsigned op, float v, float t) {
    if (op == O_DGE) return v >= t;
    if (op == O_DLE) return v <= t;
    return v == t;
}

/* Existential restriction on a numeric concrete role (Algorithms 9-10): a
 * subject belongs as soon as one of its assertions satisfies the compare. */
static void op_numeric_role(const oracle_kb *kb, unsigned op, unsigned q, float t, uint8_t *out) {
    memset(out, 0, (size_t)kb->n);
    for (int64_t k = kb->num_off[q]; k < kb->num_off[q + 1]; ++k)
        if (compare(op, kb->num_val[k], t)) out[kb->num_subj[k]] = 1;
}

static void op_data(const oracle_kb *kb, unsigned op, unsigned p, float t, uint8_t *out) {
    if ((int32_t)p >= kb->n_props) {
        op_numeric_role(kb, op, p - (unsigned)kb->n_props, t, out);
        return;
    }
    const float *v = kb->prop + (int64_t)p * kb->n;
    for (int64_t i = 0; i < kb->n; ++i) {
        if (isnan(v[i])) { out[i] = 0; continue; }
        if (op == O_DGE) out[i] = v[i] >= t;
        else if (op == O_DLE) out[i] = v[i] <= t;
        else out[i] = v[i] == t;
    }
}

static int bytes_equal(const uint8_t *x, int64_t lx, const uint8_t *y, int64_t ly) {
    if (lx != ly) return 0;
    for (int64_t i = 0; i < lx; ++i)
        if (x[i] != y[i]) return 0;
    return 1;
}

/* strContain of Algorithms 13-14: does x hold p at some position? */
static int bytes_contain(const uint8_t *x, int64_t lx, const uint8_t *p, int64_t lp) {
    for (int64_t i = 0; i + lp <= lx; ++i) {
        int64_t j = 0;
        while (j < lp && x[i + j] == p[j]) ++j;
        if (j == lp) return 1;
    }
    return 0;
}

/* Existential restriction on a string concrete role (Algorithms 11-14). */
static void op_string(const oracle_kb *kb, unsigned op, unsigned s, uint32_t b, uint8_t *out) {
    memset(out, 0, (size_t)kb->n);
    const uint8_t *y;
    int64_t ly;
    if (op == O_SEQ) {
        if ((int64_t)b >= kb->n_strings) return;   /* not in the table: nothing equals it */
        y = kb->tbl + kb->tbl_off[b];
        ly = kb->tbl_off[b + 1] - kb->tbl_off[b];
    } else {
        y = kb->pat + kb->pat_off[b];
        ly = kb->pat_off[b + 1] - kb->pat_off[b];
    }
    for (int64_t k = kb->str_off[s]; k < kb->str_off[s + 1]; ++k) {
        const uint8_t *x = kb->str_val + kb->str_val_off[k];
        const int64_t lx = kb->str_val_off[k + 1] - kb->str_val_off[k];
        if (op == O_SEQ ? bytes_equal(x, lx, y, ly) : bytes_contain(x, lx, y, ly)) out[kb->str_subj[k]] = 1;
    }
}

/* ------------------------------------------------------ byte model */
/* The algorithmic bytes of the plain method, per operation as it is
 * evaluated (no credit for sharing or caches).  A set is a row of 32-bit
 * words, W = ceil(n / 32) of them, padded to Wp = a multiple of 4, so one
 * set is B = 4 Wp bytes.  Per operation:
 *   ATOM                 B      (its row is read)
 *   TOP BOT NOT AND OR   0      (operands are counted at their leaves)
 *   role restriction     4(n+1) + 4 E_r + 2B   (row pointers, the E_r
 *                        assertions of the role, the filler written and
 *                        read; either direction)
 *   DGE DLE DEQ          4n on a one-value property; 4(n+1) + 4M on a
 *                        numeric concrete role with M assertions
 *   SEQ                  4(n+1) + 4M on a string role with M assertions
 *   SCONTAINS            the same + 4 ceil(S / 32) (the pattern's row of
 *                        the containment bitmap over the S table strings)
 *   score (per program)  2B + 16 (the example sets, four counts) */
static int64_t set_bytes(int64_t n) {
    int64_t w = (n + 31) / 32;
    int64_t wp = (w + 3) / 4 * 4;
    return 4 * wp;
}

static int64_t op_bytes(const oracle_kb *kb, uint64_t insn) {
    const unsigned op = op_of(insn), a = a_of(insn);
    const int64_t n = kb->n, B = set_bytes(n);
    switch (op) {
    case O_ATOM: return B;
    case O_TOP: case O_BOT: case O_NOT: case O_AND: case O_OR: return 0;
    case O_EXISTS: case O_FORALL: case O_ATLEAST: case O_ATMOST: case O_EXACTLY:
        return 4 * (n + 1) + 4 * (kb->role_off[a + 1] - kb->role_off[a]) + 2 * B;
    case O_DGE: case O_DLE: case O_DEQ:
        if ((int32_t)a < kb->n_props) return 4 * n;
        return 4 * (n + 1) + 4 * (kb->num_off[a - kb->n_props + 1] - kb->num_off[a - kb->n_props]);
    case O_SEQ: return 4 * (n + 1) + 4 * (kb->str_off[a + 1] - kb->str_off[a]);
    case O_SCONTAINS:
        return 4 * (n + 1) + 4 * (kb->str_off[a + 1] - kb->str_off[a]) + 4 * ((kb->n_strings + 31) / 32);
    default: return 0;
    }
}

int64_t oracle_score_bytes(int64_t n) { return 2 * set_bytes(n) + 16; }

/* Evaluate one postfix program; out receives n bytes (0/1).  With bytes != NULL
 * the algorithmic bytes of its operations are added to *bytes as they run. */
int oracle_eval_bytes(const oracle_kb *kb, const uint64_t *prog, int64_t len, uint8_t *out, int64_t *bytes);

int oracle_eval(const oracle_kb *kb, const uint64_t *prog, int64_t len, uint8_t *out) {
    return oracle_eval_bytes(kb, prog, len, out, NULL);
}

int oracle_eval_bytes(const oracle_kb *kb, const uint64_t *prog, int64_t len, uint8_t *out, int64_t *bytes) {
    int err = oracle_validate(kb, prog, len);
    if (err) return err;
    const int64_t n = kb->n;
    uint8_t *stack[ORACLE_MAX_STACK];
    int sp = 0;
    int64_t *cnt = NULL;
    uint8_t *tmp = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!tmp) return OE_NOMEM;
    for (int i = 0; i < ORACLE_MAX_STACK; ++i) stack[i] = NULL;
    for (int64_t k = 0; k < len && !err; ++k) {
        unsigned op = op_of(prog[k]);
        unsigned a = a_of(prog[k]);
        int inverse = (flags_of(prog[k]) & 1) != 0;
        int ar = arity(op);
        if (bytes) *bytes += op_bytes(kb, prog[k]);
        if (ar == 0) {
            if (!stack[sp]) stack[sp] = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
            if (!stack[sp]) { err = OE_NOMEM; break; }
            uint8_t *r = stack[sp];
            if (op == O_ATOM) memcpy(r, kb->concept_member + (int64_t)a * n, (size_t)n);
            else if (op == O_TOP) memset(r, 1, (size_t)n);
            else if (op == O_BOT) memset(r, 0, (size_t)n);
            else if (op == O_SEQ || op == O_SCONTAINS) op_string(kb, op, a, b_of(prog[k]), r);
            else op_data(kb, op, a, as_float(b_of(prog[k])), r);
            sp += 1;
        } else if (op == O_NOT) {
            uint8_t *x = stack[sp - 1];
            for (int64_t i = 0; i < n; ++i) x[i] = !x[i];
        } else if (op == O_AND || op == O_OR) {
            uint8_t *x = stack[sp - 2], *y = stack[sp - 1];
            for (int64_t i = 0; i < n; ++i) x[i] = (op == O_AND) ? (x[i] & y[i]) : (x[i] | y[i]);
            sp -= 1;
        } else {
            uint8_t *x = stack[sp - 1];
            if (op == O_EXISTS) op_exists(kb, a, inverse, x, tmp);
            else if (op == O_FORALL) op_forall(kb, a, inverse, x, tmp);
            else {
                if (!cnt) cnt = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
                if (!cnt) { err = OE_NOMEM; break; }
                op_count(kb, op, a, inverse, b_of(prog[k]), x, tmp, cnt);
            }
            memcpy(x, tmp, (size_t)n);
        }
    }
    if (!err) memcpy(out, stack[0], (size_t)n);
    for (int i = 0; i < ORACLE_MAX_STACK; ++i) free(stack[i]);
    free(tmp);
    free(cnt);
    return err;
}

/* Coverage counts of an instance set (Algorithm 15). counts = TP, FP, FN, TN. */
void oracle_score(int64_t n, const uint8_t *r, const uint8_t *pos, const uint8_t *neg, int64_t counts[4]) {
    int64_t tp = 0, fp = 0, np_ = 0, nn = 0;
    for (int64_t i = 0; i < n; ++i) {
        tp += r[i] & pos[i];
        fp += r[i] & neg[i];
        np_ += pos[i];
        nn += neg[i];
    }
    counts[0] = tp;
    counts[1] = fp;
    counts[2] = np_ - tp;
    counts[3] = nn - fp;
}

/* ------------------------------------------------------- batch, threaded */

typedef struct {
    const oracle_kb *kb;
    const uint64_t *progs;
    const int64_t *offs;
    int64_t h_begin, h_end;
    const uint8_t *pos, *neg;
    int64_t *counts;      /* [H][4] */
    uint8_t *sets;        /* [H][n] or NULL */
    int32_t *errs;        /* [H] */
    int64_t *bytes;       /* [H] or NULL: algorithmic bytes, score included */
} batch_job;

static void *batch_worker(void *arg) {
    batch_job *j = (batch_job *)arg;
    int64_t n = j->kb->n;
    uint8_t *r = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    for (int64_t h = j->h_begin; h < j->h_end; ++h) {
        uint8_t *dst = j->sets ? j->sets + h * n : r;
        int64_t b = 0;
        int e = r ? oracle_eval_bytes(j->kb, j->progs + j->offs[h], j->offs[h + 1] - j->offs[h], dst, &b) : OE_NOMEM;
        j->errs[h] = e;
        if (e == OE_OK) oracle_score(n, dst, j->pos, j->neg, j->counts + 4 * h);
        else memset(j->counts + 4 * h, 0, 4 * sizeof(int64_t));
        if (j->bytes) j->bytes[h] = e == OE_OK ? b + oracle_score_bytes(n) : 0;
    }
    free(r);
    return NULL;
}

/* Evaluate and score H programs on n_threads host threads (hypotheses split
 * into equal contiguous shares).  Returns the number of programs that failed
 * validation; their error codes are in errs.  bytes (NULL or [H]) receives
 * each program's algorithmic bytes, its score included. */
int64_t oracle_eval_batch(const oracle_kb *kb, const uint64_t *progs, const int64_t *offs, int64_t H,
                          const uint8_t *pos, const uint8_t *neg, int32_t n_threads,
                          int64_t *counts, uint8_t *sets, int32_t *errs, int64_t *bytes) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > H) n_threads = H > 0 ? (int32_t)H : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    batch_job *jobs = (batch_job *)malloc(sizeof(batch_job) * (size_t)n_threads);
    for (int32_t t = 0; t < n_threads; ++t) {
        jobs[t] = (batch_job){kb, progs, offs, H * t / n_threads, H * (t + 1) / n_threads, pos, neg,
                              counts, sets, errs, bytes};
        if (n_threads == 1) batch_worker(&jobs[t]);
        else pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    }
    if (n_threads > 1)
        for (int32_t t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
    int64_t bad = 0;
    for (int64_t h = 0; h < H; ++h) bad += errs[h] != OE_OK;
    return bad;
}
