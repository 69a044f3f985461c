/*
 * hedl.h -- C ABI of the GB300 hypothesis-evaluation library.
 *
 * The library evaluates ALCQI(D) concepts ("hypotheses") over every
 * individual of a knowledge base held in GPU memory, and scores each instance
 * set against positive and negative example sets.  It follows the paper's
 * statement of the problem (HT-HEDL, arXiv 2412.00802):
 *   - the knowledge base lives on the device for the whole session and is
 *     never copied per hypothesis (Section III-A);
 *   - a hypothesis is one contiguous array of DL operations (Section IV);
 *   - each hypothesis yields its covered positive and negative examples
 *     (Section IV, Algorithm 15), copied back once per batch (Section III-A).
 *
 * Conventions for every call:
 *   - Device pointers are CUDA global-memory addresses on the current device;
 *     host pointers are ordinary process memory.  Each parameter says which.
 *   - Device arrays passed in are BORROWED: the caller owns them, they must
 *     stay allocated and unmodified while a handle that references them is
 *     alive, and the library never frees them.  Handles (hedl_kb, hedl_plan)
 *     are owned by the library and released by their *_free call.
 *   - Work is enqueued on the given stream (NULL = the legacy default
 *     stream) and the call returns without waiting, unless the entry point
 *     says it synchronizes.  Programs are validated on the host before
 *     anything is launched, so a rejected call launches nothing.
 *   - Return value: HEDL_OK (0) or a negative hedl_status.  The calling
 *     thread's hedl_last_error() then describes the failure.  Failures found
 *     on the device (a bounded wait that gave up) are reported by the next
 *     hedl_sync_status() on the handle.
 *
 * Bitsets: a set of individuals is uint32 words, bit i of word w standing
 * for individual 32*w + i (least significant bit first).  A row has
 * hedl_row_words(n) words: ceil(n/32) rounded up to a multiple of 4, so every
 * row starts on a 16-byte boundary.  Bits of individuals >= n and padding
 * words are zero in every input and every output.
 */
#ifndef HEDL_H
#define HEDL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t. */
typedef struct CUstream_st *hedl_stream;

typedef enum {
    HEDL_OK = 0,
    HEDL_ERR_INVALID_ARG = -1,          /* a NULL / out-of-range argument */
    HEDL_ERR_BAD_PROGRAM = -2,          /* a program failed validation */
    HEDL_ERR_WORKSPACE_TOO_SMALL = -3,  /* the workspace is smaller than required */
    HEDL_ERR_CUDA = -4,                 /* a CUDA runtime call failed */
    HEDL_ERR_TIMEOUT = -5,              /* a bounded device wait gave up */
    HEDL_ERR_BAD_KB = -6,               /* the knowledge base failed validation */
    HEDL_ERR_NO_EXAMPLES = -7,          /* scoring before hedl_examples_set */
    HEDL_ERR_OOM = -8                   /* host or device allocation failed */
} hedl_status;

/*
 * Program format: postfix, one uint64 per instruction.
 *   bits  0..7   op (hedl_op)
 *   bits  8..15  flags: bit 0 = read the role inverted (r^-); other bits ignored
 *   bits 16..31  a: concept id (ATOM), role id (role ops), property id (data
 *                ops), string-role id (SEQ / SCONTAINS)
 *   bits 32..63  b: n for ATLEAST / ATMOST / EXACTLY; the IEEE float32 bit
 *                pattern of the threshold for DGE / DLE / DEQ; a string id
 *                for SEQ; a pattern id for SCONTAINS; ignored otherwise
 * AND and OR pop two operands, NOT and the role restrictions one, the rest are
 * leaves.  A valid program is non-empty, names existing ids, never pops an
 * empty stack, never holds more than HEDL_MAX_STACK operands, and leaves
 * exactly one.
 *
 * Semantics (closed world, Section III-A: what is not asserted is false):
 *   ATOM c        members of concept c
 *   TOP, BOT      every individual / no individual
 *   NOT X         the individuals not in X                      (Algs 1-2)
 *   AND, OR       intersection, union                            (Algs 1-2)
 *   EXISTS r X    a with some r-successor in X                   (Algs 3-4)
 *   FORALL r X    a all of whose r-successors are in X; an
 *                 individual without successors belongs          (Algs 5-6)
 *   ATLEAST r n X a with >= n distinct r-successors in X
 *   ATMOST r n X  a with <= n of them (zero included)
 *   EXACTLY r n X a with exactly n of them                       (Algs 7-8)
 *   r^-           subject and object swapped (Section III-B), read from
 *                 the inverse CSR
 *   DGE/DLE/DEQ   a whose value of property p is >= / <= / == t (float32
 *                 compares; a missing value, NaN, satisfies none) (Algs 9-10)
 *                 Property ids below n_props name one-value properties (a
 *                 float column); id n_props + q names numeric concrete role q
 *                 (Section III-B: a subject may assert several values), on
 *                 which the restriction is existential: a belongs as soon as
 *                 one of its values passes the compare.
 *   SEQ s v       a with a value of string role s equal to table string v;
 *                 a v outside the table matches nothing (the caller maps a
 *                 string it does not find to such an id)       (Algs 11-12)
 *   SCONTAINS s k a with a value of string role s that contains pattern k
 *                 as a substring (the empty pattern: any value) (Algs 13-14)
 */
typedef enum {
    HEDL_OP_ATOM = 1, HEDL_OP_TOP = 2, HEDL_OP_BOT = 3, HEDL_OP_NOT = 4,
    HEDL_OP_AND = 5, HEDL_OP_OR = 6,
    HEDL_OP_EXISTS = 7, HEDL_OP_FORALL = 8, HEDL_OP_ATLEAST = 9, HEDL_OP_ATMOST = 10,
    HEDL_OP_EXACTLY = 11,
    HEDL_OP_DGE = 12, HEDL_OP_DLE = 13, HEDL_OP_DEQ = 14,
    HEDL_OP_SEQ = 15, HEDL_OP_SCONTAINS = 16
} hedl_op;

#define HEDL_FLAG_INVERSE 1u
#define HEDL_MAX_STACK 64

/* Words per bitset row for n individuals: ceil(n/32) rounded up to 4. */
uint32_t hedl_row_words(uint32_t n_indiv);

/* ------------------------------------------------------------------ KB */

/* One role's assertions as CSR (rows = subjects, Section III-A's 2-column
 * role matrix grouped by subject). Device arrays: row_ptr uint32[n_indiv+1]
 * with row_ptr[0] = 0 and row_ptr[n_indiv] = n_edges; col uint32[n_edges],
 * each row strictly increasing (a set of distinct objects < n_indiv). */
typedef struct {
    const uint32_t *row_ptr;
    const uint32_t *col;
    uint32_t n_edges;          /* < 2^31 */
} hedl_csr;

/* One numeric concrete role (Section III-B): the (subject, value) assertions
 * grouped by subject as CSR.  Device arrays: row_ptr uint32[n_indiv+1] with
 * row_ptr[0] = 0, non-decreasing, row_ptr[n_indiv] = n_vals; vals
 * float32[n_vals], subject i's values at vals[row_ptr[i] .. row_ptr[i+1]) in
 * any order (duplicates allowed; a NaN value satisfies no compare). */
typedef struct {
    const uint32_t *row_ptr;
    const float *vals;
    uint32_t n_vals;           /* < 2^31 */
} hedl_numeric_role;

/* One string concrete role (Section III-B): the (subject, string) assertions
 * grouped by subject as CSR of interned string ids.  Device arrays: row_ptr
 * uint32[n_indiv+1] as for hedl_numeric_role; ids uint32[n_vals], each below
 * the descriptor's n_strings. */
typedef struct {
    const uint32_t *row_ptr;
    const uint32_t *ids;
    uint32_t n_vals;           /* < 2^31 */
} hedl_string_role;

typedef struct {
    uint32_t n_indiv;                  /* individuals, >= 1 */
    uint32_t n_concepts;
    const uint32_t *concept_bits;      /* device, [n_concepts][hedl_row_words(n)] */
    uint32_t n_roles;
    const hedl_csr *roles;             /* HOST array [n_roles] of device CSRs */
    const hedl_csr *inv_roles;         /* HOST array [n_roles]: the transposes */
    uint32_t n_props;
    const float *prop_vals;            /* device, [n_props][prop_stride], NaN = missing */
    uint64_t prop_stride;              /* floats between property rows, >= n_indiv */
    uint32_t n_num_roles;              /* numeric concrete roles: property ids n_props + q */
    const hedl_numeric_role *num_roles;/* HOST array [n_num_roles] of device CSRs */
    uint32_t n_str_roles;              /* string concrete roles: ids of SEQ / SCONTAINS */
    const hedl_string_role *str_roles; /* HOST array [n_str_roles] of device CSRs */
    uint32_t n_strings;                /* the string table: DISTINCT strings (interned) */
    const uint32_t *str_off;           /* device [n_strings+1]: string i is chars [off[i], off[i+1]) */
    const uint8_t *str_chars;          /* device [n_str_chars] */
    uint32_t n_str_chars;
    uint32_t n_patterns;               /* substring patterns of SCONTAINS, fixed for the handle */
    const uint32_t *pat_off;           /* HOST [n_patterns+1] */
    const uint8_t *pat_chars;          /* HOST [pat_off[n_patterns]] */
} hedl_kb_desc;

typedef struct hedl_kb hedl_kb;

#define HEDL_KB_NO_VALIDATE 1u   /* skip the device-side structural checks */

/* Register a knowledge base resident on the device (Section III-A).
 * Borrows every device array of d (see the conventions above); copies the
 * small host arrays roles / inv_roles / num_roles / str_roles and the
 * patterns (to the device).  n_props + n_num_roles and n_str_roles are at most
 * 65536 (16-bit ids).  Unless HEDL_KB_NO_VALIDATE, checks on the device that
 * concept rows have zero tails, that each CSR is well formed (monotone
 * row_ptr, rows strictly increasing, ids < n), that each inverse CSR is
 * exactly the transpose of its forward CSR, that each numeric and string
 * role's row_ptr starts at 0, never decreases and ends at n_vals, that string
 * ids are below n_strings and that str_off starts at 0, never decreases and
 * ends at n_str_chars; a failed check returns HEDL_ERR_BAD_KB and no handle.
 * With HEDL_KB_NO_VALIDATE the caller guarantees all of that.  That the table
 * holds distinct strings is never checked: SEQ compares ids.  Then computes,
 * on the device, which table strings contain which pattern (a bitmap the
 * handle owns; SCONTAINS reads it).  SYNCHRONIZES the stream.
 * *out receives the handle; release it with hedl_kb_free. */
int hedl_kb_load(const hedl_kb_desc *d, unsigned flags, hedl_stream s, hedl_kb **out);

/* A planning-only handle: reads only the sizes in d (n_indiv, the counts,
 * each role's n_edges and each numeric and string role's n_vals; device
 * pointers may be NULL; patterns are not read) and makes no CUDA call, so it
 * works on a host without a GPU.  hedl_validate, hedl_plan_batch and
 * hedl_plan_info_get accept it (its plans are shaped for a 152-SM GB300);
 * every call that would launch work returns HEDL_ERR_INVALID_ARG.  Release
 * it with hedl_kb_free. */
int hedl_kb_plan_only(const hedl_kb_desc *d, hedl_kb **out);

/* Release a handle (waits for the device to go idle first).  NULL is fine. */
void hedl_kb_free(hedl_kb *kb);

/* Set the positive and negative examples (Section IV's examples matrix) as
 * two borrowed device bitsets of hedl_row_words(n) words each.  Computes |P|
 * and |N| on the device.  SYNCHRONIZES the stream.  Until it is called,
 * scoring entry points return HEDL_ERR_NO_EXAMPLES. */
int hedl_examples_set(hedl_kb *kb, const uint32_t *pos_bits, const uint32_t *neg_bits, hedl_stream s);

/* |P| and |N| as cached by hedl_examples_set (host values). */
int hedl_examples_counts(const hedl_kb *kb, uint32_t *n_pos, uint32_t *n_neg);

/* Host-only validation of one program against the KB's ids (no GPU work).
 * Returns HEDL_OK or HEDL_ERR_BAD_PROGRAM (reason in hedl_last_error). */
int hedl_validate(const hedl_kb *kb, const uint64_t *prog, uint32_t len);

/* ------------------------------------------------------------------ plans */

/* A batch of programs compiled on the host into a device work queue: the
 * programs' expression DAG with common sub-concepts shared across the batch
 * (hash-consing), cut into segments at role restrictions (a role restriction
 * needs its filler over all individuals before any tile of its result), each
 * segment split into tiles of individuals.  The paper builds one evaluation
 * plan per hypothesis on the CPU (Section IV; multi-threaded, Section V). */
typedef struct hedl_plan hedl_plan;

#define HEDL_NO_CSE     1u   /* no sharing of common sub-concepts */
#define HEDL_NO_GRAPH   2u   /* always launch directly (default: a plan's first execution
                                launches directly, later ones capture and then replay a
                                CUDA graph) */
#define HEDL_PLAIN      4u   /* one launch per operation per hypothesis */
#define HEDL_LEVELS     8u   /* one launch per dependency level, no device waits */
#define HEDL_NO_SLICE  16u   /* evaluate every role restriction on its own CSR walk
                                (default: up to 32 restrictions of one role and
                                direction that become ready together share one walk,
                                formed where at least two restrictions have the same
                                role, direction and nesting depth of role restrictions) */
#define HEDL_SLICE_ALL 32u   /* put every eligible role restriction in a shared walk,
                                even a group of one (ignored with HEDL_NO_SLICE) */
#define HEDL_TEST_UNSAT_DEP 0x100u  /* TEST HOOK: add a dependency nothing
                                        satisfies, so the bounded device wait
                                        gives up (the call then reports
                                        HEDL_ERR_TIMEOUT) */

typedef struct {
    uint32_t n_hyps;
    uint32_t n_nodes;        /* distinct DAG nodes after sharing */
    uint32_t n_segments;
    uint32_t n_slots;        /* materialized intermediate bitsets */
    uint32_t n_levels;
    uint32_t n_items;        /* (segment, tile) work items */
    uint32_t tile_words;
    uint32_t n_role_ops;     /* role restrictions evaluated (after sharing) */
    uint32_t n_role_groups;  /* shared CSR walks of bit-sliced role restrictions */
    uint32_t n_data_ops;
    uint32_t n_atom_loads;
    uint32_t warp_words;     /* words a warp covers per round: 32, or 16 / 8 / 4 when a
                                level walking a role has too few segments to fill the GPU
                                (0 with HEDL_PLAIN, which has no tiles) */
    uint64_t total_insns;    /* instructions in the input programs */
    uint64_t workspace_bytes;
    uint64_t image_bytes;    /* plan image copied host-to-device by hedl_plan_execute */
    uint64_t model_bytes;    /* algorithmic bytes of the plan (one pass) */
} hedl_plan_info;

/* Compile H programs (HOST arrays: progs uint64[offs[H]], offs uint32[H+1],
 * program h = progs[offs[h] .. offs[h+1])).  Rejects the batch with
 * HEDL_ERR_BAD_PROGRAM naming the first bad program.  Host-only; the plan
 * keeps no pointer to the inputs. */
int hedl_plan_batch(const hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H,
                    unsigned flags, hedl_plan **out);
int hedl_plan_info_get(const hedl_plan *p, hedl_plan_info *info);
void hedl_plan_free(hedl_plan *p);

/* The same plan as hedl_plan_batch with HEDL_NO_CSE | HEDL_NO_SLICE (no
 * sharing of sub-concepts, no bit slicing), built one hypothesis at a time on
 * n_threads host threads (0 = one per hardware thread): the paper plans the
 * hypotheses of a batch in parallel on the CPU (Section V).  Every
 * per-hypothesis step is independent and every global one a prefix sum, a
 * reduction or a stable sort, the form a device-side planner takes.  The
 * image equals hedl_plan_batch's for those flags, byte for byte.  flags may
 * add HEDL_NO_GRAPH or HEDL_LEVELS; HEDL_PLAIN and HEDL_SLICE_ALL are refused
 * (HEDL_ERR_INVALID_ARG), and so is a batch whose plan would have more than
 * 16,384 dependency levels (a chain of that many nested role restrictions),
 * which hedl_plan_batch still plans.  Host-only; HOST progs / offs as in
 * hedl_plan_batch. */
int hedl_plan_batch_parallel(const hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H,
                             unsigned flags, uint32_t n_threads, hedl_plan **out);

/* The same plan built on the device (the paper's future work, Section VII:
 * the GPU generates its own evaluation plans): the per-hypothesis steps of
 * hedl_plan_batch_parallel run as grid-stride kernels over DEVICE programs
 * (progs uint64[n_insns], offs uint32[H+1], offs[0] = 0, offs[H] = n_insns),
 * the prefix sums as block-wide scans, the work-queue order as a bitonic
 * sort.  Validation runs on the device too (HEDL_ERR_BAD_PROGRAM names the
 * first bad program; offsets outside [0, n_insns] or decreasing give
 * HEDL_ERR_INVALID_ARG).  The image (byte for byte hedl_plan_batch's with
 * HEDL_NO_CSE | HEDL_NO_SLICE) stays in device memory owned by the plan;
 * hedl_plan_execute copies it into the workspace within the device, and
 * hedl_plan_image copies it to the host.  The library allocates the planner's
 * scratch (about 80 bytes per instruction) for the call and the image for the
 * plan's lifetime.  Flags and the depth limit as hedl_plan_batch_parallel.
 * Synchronizes s twice (the totals size the image; the header comes back). */
int hedl_plan_batch_device(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, uint64_t n_insns,
                           unsigned flags, hedl_stream s, hedl_plan **out);

/* Copy a plan's image (the work queue the interpreter reads: header, task and
 * group tables, dependency lists, segment code, zeroed counters; image_bytes
 * of hedl_plan_info) into the HOST buffer out of cap bytes, and its size into
 * *bytes.  For inspection and tests; the layout is the library's own and may
 * change with it.  A HEDL_PLAIN plan has no image (size 0).  Returns
 * HEDL_ERR_INVALID_ARG if cap is smaller than the image (with *bytes set). */
int hedl_plan_image(const hedl_plan *p, void *out, size_t cap, size_t *bytes);

/* Execute a plan.  counts: device uint32[H][4] receiving (TP, FP, FN, TN) per
 * program (Algorithm 15 and its complements), or NULL; out_bits: device
 * uint32[H][hedl_row_words(n)] receiving each instance set, or NULL (not both
 * NULL).  ws: device workspace of ws_bytes >= workspace_bytes of the plan
 * info, 256-byte aligned, used exclusively by this call until it completes.
 * The plan image is copied host-to-device on s.  Asynchronous. */
int hedl_plan_execute(hedl_kb *kb, const hedl_plan *p, uint32_t *counts, uint32_t *out_bits,
                      void *ws, size_t ws_bytes, hedl_stream s);

/* Run again a plan whose image an earlier hedl_plan_execute on the same ws
 * already put there (ws not reused since): only the plan's counters are
 * reset, nothing is copied from the host.  Same arguments as
 * hedl_plan_execute.  Asynchronous. */
int hedl_plan_replay(hedl_kb *kb, const hedl_plan *p, uint32_t *counts, uint32_t *out_bits,
                     void *ws, size_t ws_bytes, hedl_stream s);

/* ------------------------------------------------------------------ one-shot calls */

/* Workspace bytes hedl_score_batch / hedl_eval_concept need for these
 * programs and flags (plans them; the plan is cached on the handle so the
 * following call with the same programs does not plan again). */
int hedl_workspace_size(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H,
                        unsigned flags, size_t *bytes);

/* Evaluate and score H programs (HOST progs/offs as in hedl_plan_batch) into
 * device counts uint32[H][4] = (TP, FP, FN, TN).  Plans (or reuses the cached
 * plan), copies the plan image to ws and launches.  Asynchronous. */
int hedl_score_batch(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H,
                     uint32_t *counts, void *ws, size_t ws_bytes, unsigned flags, hedl_stream s);

/* Evaluate one program (HOST prog uint64[len]) into the device bitset
 * out_bits (hedl_row_words(n) words).  Workspace as for hedl_score_batch with
 * H = 1.  Asynchronous. */
int hedl_eval_concept(hedl_kb *kb, const uint64_t *prog, uint32_t len, uint32_t *out_bits,
                      void *ws, size_t ws_bytes, unsigned flags, hedl_stream s);

/* Size of the scratch array built into the library for
 * hedl_eval_concept_noalloc (device memory held on every GPU that loads the
 * library, until the process exits). */
#define HEDL_NOALLOC_SCRATCH_BYTES (16u << 20)

/* hedl_eval_concept without a caller workspace and without allocating: for
 * callers that cannot call cudaMalloc (or any device allocator) when they
 * evaluate, and so cannot provide the workspace hedl_eval_concept needs.  The
 * paper has no counterpart; this is a deployment convenience.
 *   - Scratch: a fixed HEDL_NOALLOC_SCRATCH_BYTES device array inside the
 *     library; a program whose plan needs more (hedl_workspace_size with H = 1
 *     and flags HEDL_NO_GRAPH tells) is rejected with
 *     HEDL_ERR_WORKSPACE_TOO_SMALL before anything is launched.
 *   - Set-up: the first call on each device (that device current) looks up
 *     the array's device address and remembers it with the device's current
 *     context; after cudaDeviceReset the next call looks it up again.  Make
 *     the first call on a device, and the first after a reset, before any
 *     stream capture.
 *   - Sharing: every call uses the same array and brings its own zeroed
 *     counters, so nothing carries over between calls; calls whose GPU work
 *     overlaps race on the array and must be ordered by the caller.
 *   - Calls no cudaMalloc / cudaFree or other allocating routine, and builds no
 *     CUDA graph.
 * prog (HOST uint64[len]) and out_bits (device, hedl_row_words(n) words) as in
 * hedl_eval_concept.  Asynchronous. */
int hedl_eval_concept_noalloc(hedl_kb *kb, const uint64_t *prog, uint32_t len, uint32_t *out_bits,
                              hedl_stream s);

/* Wait for s, then report (and clear) the first device-side failure recorded
 * by work launched on this handle since the last call: HEDL_OK,
 * HEDL_ERR_TIMEOUT, or HEDL_ERR_CUDA for an asynchronous CUDA error. */
int hedl_sync_status(hedl_kb *kb, hedl_stream s);

/* ------------------------------------------------------------------ tuning */

typedef struct {
    uint32_t warps_per_cta;    /* 1, 2, 4, 8, 16 or 32 (1 and 2: one word per lane, no
                                  staging; a CTA's warps share each work item, so small
                                  CTAs wait less on their slowest warp) */
    uint32_t words_per_lane;   /* 1 or 4: bitset words a lane holds per pass */
    uint32_t rounds;           /* warp passes per work item (tile = warps*32*words_per_lane*rounds words) */
    uint32_t ctas_per_sm;      /* 0 = as many as fit */
    uint32_t wait_timeout_ms;  /* bound of every device-side dependency wait */
    uint32_t stage_fillers;    /* 1: copy a role restriction's filler row into shared memory once per
                                  work item when it fits (then a segment reads at most one role
                                  restriction); 0: gather filler bits from global memory */
    uint32_t role_block;       /* 4 or 8: 32-edge chunks the role walk loads per step */
    uint32_t full_occupancy;   /* 1: with 8 warps, 1 word per lane and no staging, use the build
                                  limited to 32 registers so 8 CTAs fit per SM */
} hedl_tuning;

int hedl_tuning_get(const hedl_kb *kb, hedl_tuning *t);
/* Set the launch shape used by later plans and executions on this handle;
 * rejects unsupported values with HEDL_ERR_INVALID_ARG. */
int hedl_tuning_set(hedl_kb *kb, const hedl_tuning *t);

/* Workspace bytes hedl_autotune needs for this probe batch: the largest plan
 * over every candidate launch shape.  Host-only. */
int hedl_autotune_workspace_size(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H,
                                 size_t *bytes);

/* Autotuner for the launch shape (warps per CTA, words per lane, rounds per
 * work item, chunks per role-walk step, filler staging).  No counterpart in
 * the paper.  Each candidate shape plans the probe batch (HOST progs / offs as
 * in hedl_plan_batch, scored against the handle's examples), runs it once,
 * then times three replays with CUDA events on s; the fastest becomes the
 * handle's tuning and is written to *chosen (may be NULL), except that the
 * handle's current shape is kept when it is within 2 % of the fastest (so
 * timing noise between near-equal shapes does not flip the choice).  With cache_path
 * (may be NULL), a result stored earlier for the same KB shape and GPU is
 * reused without timing, and a new result is appended to that text file.
 * ws (>= hedl_autotune_workspace_size, 256-byte aligned) is scratch for the
 * duration of the call.  SYNCHRONIZES s.  On failure the tuning is unchanged. */
int hedl_autotune(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, void *ws,
                  size_t ws_bytes, const char *cache_path, hedl_stream s, hedl_tuning *chosen);

/* ------------------------------------------------------------------ refinement search */

/* Canonical form of H programs (HOST arrays as in hedl_plan_batch) for the
 * beam search's duplicate removal (the paper has no search loop): every AND /
 * OR gets its two operands in ascending order of their canonical instruction
 * bytes (the little-endian instruction words compared byte by byte, a proper
 * prefix first); everything else keeps its place.  out (HOST uint64[offs[H]],
 * may alias progs) receives the programs at the same offsets.  Host-only.
 * HEDL_ERR_BAD_PROGRAM names the first program that is not a valid postfix
 * program. */
int hedl_canonical_batch(const uint64_t *progs, const uint32_t *offs, uint32_t H, uint64_t *out);

/* ------------------------------------------------------------------ surrogate */
/* A learned surrogate that predicts a hypothesis' (accuracy, F1) from a
 * structural encoding, used only to order and prune the queue of exact
 * evaluations; every reported score still comes from exact evaluation.  The
 * paper has no learned component.  Network: 512 -> 512 -> 512 -> 2, ReLU,
 * BF16 weights and activations, FP32 accumulation on the tensor cores;
 * trained by mean squared error with Adam on FP32 master weights. */
typedef struct hedl_mlp hedl_mlp;

#define HEDL_ENC_DIM 512
#define HEDL_ENC_MAXLEN 256   /* longer programs are encoded by their last 256 instructions */

/* Number of parameters: W1[512][512], b1[512], W2[512][512], b2[512],
 * W3[2][512], b3[2], concatenated in that order (row-major). */
uint64_t hedl_mlp_param_count(void);

/* Create a network from HOST params (float32[hedl_mlp_param_count()]).
 * Allocates its device state; SYNCHRONIZES the device. */
int hedl_mlp_create(const float *params, hedl_mlp **out);
void hedl_mlp_free(hedl_mlp *m);

/* Copy the FP32 master weights and/or the last gradients (HOST arrays of
 * hedl_mlp_param_count() floats, either may be NULL) and the Adam step count.
 * SYNCHRONIZES the device. */
int hedl_mlp_get(const hedl_mlp *m, float *params, float *grads, uint32_t *step);

/* Copy the Adam moments (HOST float [hedl_mlp_param_count()] each, either may
 * be NULL): the first moment m and the second moment v of Adam's definition
 * (Kingma and Ba, 2015), as left by the last hedl_mlp_train_step, zero before
 * the first.  The paper has no learned component: for checking the optimiser.
 * SYNCHRONIZES the device. */
int hedl_mlp_get_moments(const hedl_mlp *m, float *first, float *second);

/* Workspace bytes for a batch of B rows (activations and their gradients). */
int hedl_mlp_workspace_size(uint32_t B, size_t *bytes);

/* Structural encoding of H programs (DEVICE progs uint64[offs[H]], offs
 * uint32[H+1]) into X (DEVICE bf16 [H][512] as uint16 bit patterns).  The
 * paper has no learned component: this is the surrogate's input.  Features
 * 0..509 are integer counts scaled by 1/4: op histogram per depth, atomic
 * concepts, roles, restriction kinds per depth, cardinalities, >= / <=
 * restrictions by property and threshold bucket, role-over-atom pairs,
 * length, sums of the symbols' statistics, totals, a constant; concepts,
 * thresholds, role-over-atom pairs and statistics count -1 at odd polarity
 * (under an odd number of NOT / ATMOST).  grid (DEVICE float [n_grid][15],
 * or NULL) holds each property's 15 increasing threshold boundaries: a
 * threshold t of property p lands in bucket q = #{g < t}.  stats (DEVICE
 * int32, or NULL for zeros) holds n_stat_concepts atom scores, then
 * n_grid x 2 x 16 scores of (property, >= / <=, bucket), as written by
 * hedl_stat_scores from the engine's exact scores of those symbols.  prior
 * (DEVICE float [H][2], or NULL for zeros) gives features 510-511 per
 * program, rounded to bf16 (the search passes the exact accuracy and F1 of
 * the hypothesis a candidate refines).  Instructions that are not op codes
 * are ignored.  Asynchronous. */
int hedl_encode(const uint64_t *progs, const uint32_t *offs, uint32_t H, const float *grid, uint32_t n_grid,
                const int32_t *stats, uint32_t n_stat_concepts, const float *prior, uint16_t *X, hedl_stream s);

/* Statistics table entries (DEVICE int32 [n]) from exact scores (DEVICE
 * float [n][2], accuracy first): round((accuracy - 1/2) * 32), computed in
 * double, ties to even.  Asynchronous. */
int hedl_stat_scores(const float *scores, uint32_t n, int32_t *out, hedl_stream s);

/* Engine of the 512-wide dense layers' GEMMs: HEDL_GEMM_TCGEN05 (default)
 * runs the forward layers, and the backward pass's weight and activation
 * gradients when the batch is a multiple of 64, on the 5th-generation tensor
 * cores (tcgen05.mma, accumulators in tensor memory); HEDL_GEMM_MMA_SYNC on
 * the warp-level mma.sync path.  Both accumulate in FP32 and store bf16
 * activations and activation gradients. */
#define HEDL_GEMM_TCGEN05  0u
#define HEDL_GEMM_MMA_SYNC 1u
int hedl_mlp_set_gemm(hedl_mlp *m, unsigned engine);

/* SYNCHRONIZES the stream; HEDL_ERR_TIMEOUT if a tensor-core completion wait
 * of an earlier call gave up (its outputs are then undefined), and clears it. */
int hedl_mlp_status(hedl_mlp *m, hedl_stream s);

/* Y (DEVICE float [B][2]) = the network applied to X (DEVICE bf16 [B][512]),
 * its raw output u mapped to the target scale: Y = u * scale + mean (the
 * target map; identity until one is set). */
int hedl_mlp_forward(hedl_mlp *m, const uint16_t *X, uint32_t B, float *Y, void *ws, size_t ws_bytes,
                     hedl_stream s);

/* Gradients of the loss mean_b w_b sum_j (u_bj - t_bj)^2, where u is the raw
 * output, t = (T - mean) / scale the mapped targets T (DEVICE float [B][2])
 * and w_b = 1 + tail * max(0, t_b0) (the upper tail of the first target
 * weighs more), into the network's gradient buffer; *loss (DEVICE float, may
 * be NULL) receives the loss.  With the identity map this is the plain mean
 * squared error. */
int hedl_mlp_gradients(hedl_mlp *m, const uint16_t *X, const float *T, uint32_t B, float *loss, void *ws,
                       size_t ws_bytes, hedl_stream s);

/* hedl_mlp_gradients followed by one Adam step (beta 0.9 / 0.999, eps 1e-8,
 * learning rate lr) on the master weights, refreshing their BF16 copies. */
int hedl_mlp_train_step(hedl_mlp *m, const uint16_t *X, const float *T, uint32_t B, float lr, float *loss,
                        void *ws, size_t ws_bytes, hedl_stream s);

/* Target map (mean0, mean1, scale0, scale1, tail weight) of a network.
 * fit: means and population standard deviations (1 where below 1e-6) of the
 * columns of T (DEVICE float [B][2], B >= 1), and tail_weight >= 0;
 * asynchronous.  set / get: HOST float[5]; scales must be > 0; SYNCHRONIZE.
 * The map standardises the training targets and maps predictions back. */
int hedl_mlp_fit_target_map(hedl_mlp *m, const float *T, uint32_t B, float tail_weight, hedl_stream s);
int hedl_mlp_set_target_map(hedl_mlp *m, const float *map);
int hedl_mlp_get_target_map(const hedl_mlp *m, float *map);

/* Exact scores from coverage counts (DEVICE uint32 [H][4] TP, FP, FN, TN) into
 * DEVICE float [H][2]: accuracy (TP+TN)/(TP+FP+FN+TN) and F1 2TP/(2TP+FP+FN)
 * (0 where the denominator is 0), computed in double, stored as float. */
int hedl_scores_from_counts(const uint32_t *counts, uint32_t H, float *scores, hedl_stream s);

/* Indices (DEVICE uint32 [k], ascending) of the k best rows of Y (DEVICE
 * float [H][2]) ordered by Y[.][0] descending, then Y[.][1] descending, then
 * index ascending (NaN last).  ws >= hedl_select_workspace_size(H). */
int hedl_select_workspace_size(uint32_t H, size_t *bytes);
int hedl_select_top(const float *Y, uint32_t H, uint32_t k, uint32_t *idx, void *ws, size_t ws_bytes,
                    hedl_stream s);

/* Description of the calling thread's last failure ("" if none). */
const char *hedl_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HEDL_H */
