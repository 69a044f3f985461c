// Plans without sharing or bit slicing, built one hypothesis at a time.
//
// These are the host planner's steps (plan.cpp) for HEDL_NO_CSE | HEDL_NO_SLICE
// (role fillers staged or not), written so that every per-hypothesis step is a
// __host__ __device__ function over that hypothesis's instructions and its own
// stretch of scratch, and every global step is a prefix sum, a reduction or a
// stable sort:
//   1. per hypothesis: the expression tree (one node per instruction), the
//      materialised nodes (role fillers that are not a concept, and the larger
//      operand wherever an AND / OR would need more than STACK_MAX - 1 stack
//      entries), each node's stack need (Sethi-Ullman);
//   2. per hypothesis: each segment (one per materialised node, in node order,
//      then the root) counted, then emitted in post-order with the larger-need
//      operand first, with the slots it reads, its level (one above them), its
//      first role restriction's key, its staged filler, its algorithmic bytes;
//   3. prefix sums over hypotheses: slot ids, segment ids, code and dependency
//      offsets;
//   4. a reduction (segments per level that walk a role) fixes the tile shape
//      and a stable sort by (level, role key) orders the work queue.
// The host driver runs the per-hypothesis steps on several threads (the paper
// plans hypotheses in parallel on the CPU, Section V) and the others in turn;
// every step is a __host__ __device__ function of one index, so the same code
// is the body of a device-side planner (the paper's future work, Section VII).
// The image equals the host planner's for the same flags, byte for byte.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>
#include <thread>
#include <vector>

#include "hedl_internal.h"

namespace hedl {
namespace dp {

__host__ __device__ inline uint32_t op_of(uint64_t w) { return (uint32_t)(w & 0xFF); }
__host__ __device__ inline uint32_t a_of(uint64_t w) { return (uint32_t)((w >> 16) & 0xFFFF); }
__host__ __device__ inline uint32_t b_of(uint64_t w) { return (uint32_t)(w >> 32); }
__host__ __device__ inline uint32_t inv_of(uint64_t w) { return (uint32_t)((w >> 8) & 1); }
__host__ __device__ inline bool is_role(uint32_t op) { return op >= HEDL_OP_EXISTS && op <= HEDL_OP_EXACTLY; }
__host__ __device__ inline bool is_count(uint32_t op) { return op >= HEDL_OP_ATLEAST && op <= HEDL_OP_EXACTLY; }
__host__ __device__ inline bool is_data(uint32_t op) { return op >= HEDL_OP_DGE && op <= HEDL_OP_DEQ; }
__host__ __device__ inline bool is_str(uint32_t op) { return op == HEDL_OP_SEQ || op == HEDL_OP_SCONTAINS; }
__host__ __device__ inline int arity(uint32_t op) {
    if (op == HEDL_OP_NOT || is_role(op)) return 1;
    if (op == HEDL_OP_AND || op == HEDL_OP_OR) return 2;
    return 0;
}

// What a plan needs to know of the KB (plain pointers, copyable to the device).
struct Sizes {
    uint64_t N, B;                  // individuals, bytes per bitset row
    uint32_t n_props;               // one-value properties (numeric roles follow)
    const uint32_t *num_vals;       // [numeric roles] values
    const uint32_t *str_vals;       // [string roles] values
    const uint32_t *csr_edges;      // [2 * roles] edges of role r forward (2r) and inverse (2r + 1)
    uint64_t contain_words;         // words of a pattern's containment row
};

// Scratch indexed by global instruction position; a hypothesis uses only its
// own stretch [o0, o1), so hypotheses run independently.
struct Scratch {
    int32_t *k0, *k1;     // operands (instruction positions), -1 for none
    uint32_t *need;       // stack need of the node's expression
    uint8_t *mat;         // materialised into a slot
    uint32_t *slot;       // local slot id of a materialised node
    uint32_t *level;      // level of a materialised node's segment
    uint32_t *stk;        // the tree build's operand stack, then emission frames
    uint8_t *state;       // emission frame states
};

// Step 1.  Returns the root's position.  The program is valid (validated).
// staged: role fillers are staged in shared memory, one role restriction per
// segment, so every further role restriction met in a segment's inline
// expansion (depth-first, first operand first) is materialised as well.
__host__ __device__ inline uint32_t analyze(const uint64_t *progs, uint32_t o0, uint32_t o1, const Scratch &sc,
                                            bool staged) {
    uint32_t sp = 0;
    for (uint32_t k = o0; k < o1; ++k) {
        const int ar = arity(op_of(progs[k]));
        int32_t x = -1, y = -1;
        if (ar == 2) {
            y = (int32_t)sc.stk[o0 + --sp];
            x = (int32_t)sc.stk[o0 + --sp];
        } else if (ar == 1) {
            x = (int32_t)sc.stk[o0 + --sp];
        }
        sc.k0[k] = x;
        sc.k1[k] = y;
        sc.mat[k] = 0;
        sc.need[k] = 1;
        sc.stk[o0 + sp++] = k;
    }
    const uint32_t root = sc.stk[o0];
    for (uint32_t k = o0; k < o1; ++k)
        if (is_role(op_of(progs[k])) && op_of(progs[sc.k0[k]]) != HEDL_OP_ATOM) sc.mat[sc.k0[k]] = 1;
    for (uint32_t k = o0; k < o1; ++k) {
        const uint32_t op = op_of(progs[k]);
        const int32_t x = sc.k0[k], y = sc.k1[k];
        if (op == HEDL_OP_NOT) {
            sc.need[k] = sc.mat[x] ? 1u : sc.need[x];
        } else if (op == HEDL_OP_AND || op == HEDL_OP_OR) {
            uint32_t a = sc.mat[x] ? 1u : sc.need[x], b = sc.mat[y] ? 1u : sc.need[y];
            uint32_t v = a == b ? a + 1 : (a > b ? a : b);
            if (v > (uint32_t)STACK_MAX - 1) {   // keep every segment within the device stack
                sc.mat[a >= b ? x : y] = 1;
                a = sc.mat[x] ? 1u : sc.need[x];
                b = sc.mat[y] ? 1u : sc.need[y];
                v = a == b ? a + 1 : (a > b ? a : b);
            }
            sc.need[k] = v;
        }
    }
    if (staged) {
        for (uint32_t q = o0; q <= o1; ++q) {   // segment roots: materialised nodes, then the root
            const uint32_t r = q < o1 ? q : root;
            if (q < o1 && !sc.mat[r]) continue;
            if (q == o1 && sc.mat[r]) continue;
            bool kept = false;
            uint32_t sp2 = 0;
            sc.stk[o0 + sp2++] = r;
            while (sp2) {
                const uint32_t i = sc.stk[o0 + --sp2];
                if (i != r && sc.mat[i]) continue;
                if (is_role(op_of(progs[i]))) {
                    if (kept && i != r) sc.mat[i] = 1;
                    kept = true;
                    continue;   // its filler is a slot or a concept row, not inline
                }
                if (sc.k1[i] >= 0) sc.stk[o0 + sp2++] = (uint32_t)sc.k1[i];
                if (sc.k0[i] >= 0) sc.stk[o0 + sp2++] = (uint32_t)sc.k0[i];
            }
        }
    }
    return root;
}

// One segment's summary.
struct SegInfo {
    uint32_t code_len = 0, n_reads = 0, level = 0, key = NO_FILLER, filler = NO_FILLER, max_depth = 0;
    uint32_t n_role = 0, n_data = 0, n_atom = 0;
    uint64_t model = 0;
};

// Step 2 for the segment rooted at `root`: counts it, and with code != nullptr
// also writes its code and the (global) slots it reads.  slot_base: the
// hypothesis's first global slot id.
__host__ __device__ inline SegInfo emit(const uint64_t *progs, uint32_t o0, const Scratch &sc, uint32_t root,
                                        const Sizes &z, uint32_t slot_base, DInsn *code, uint32_t *reads) {
    SegInfo s;
    uint32_t fp = 0;   // frames: node at stk[o0 + f], state at state[o0 + f]
    sc.stk[o0] = root;
    sc.state[o0] = 0;
    fp = 1;
    uint32_t depth = 0;
    auto put = [&](uint32_t op, uint32_t a, uint32_t b, uint32_t ref) {
        if (code) code[s.code_len] = DInsn{op, a, b, ref};
        s.code_len++;
    };
    auto read = [&](uint32_t node) {
        const uint32_t g = slot_base + sc.slot[node];
        if (reads) reads[s.n_reads] = g;
        s.n_reads++;
        if (sc.level[node] + 1 > s.level) s.level = sc.level[node] + 1;
        return g;
    };
    while (fp) {
        const uint32_t i = sc.stk[o0 + fp - 1];
        const uint64_t w = progs[i];
        const uint32_t op = op_of(w);
        if ((i != root && sc.mat[i]) || arity(op) == 0 || is_role(op)) {
            if (i != root && sc.mat[i]) {
                put(D_SLOT, 0, 0, read(i));
            } else if (op == HEDL_OP_ATOM) {
                put(D_ATOM, a_of(w), 0, 0);
                s.model += z.B;
                s.n_atom++;
            } else if (op == HEDL_OP_TOP || op == HEDL_OP_BOT) {
                put(op, 0, 0, 0);
            } else if (is_data(op)) {
                const uint32_t a = a_of(w);
                const bool num = a >= z.n_props;
                put(D_DATA | (op << 16) | (num ? 1u << 8 : 0u), num ? a - z.n_props : a, b_of(w), 0);
                s.model += num ? 4 * (z.N + 1) + 4ull * z.num_vals[a - z.n_props] : 4 * z.N;
                s.n_data++;
            } else if (is_str(op)) {
                const uint32_t a = a_of(w);
                put(D_DATA | (op << 16) | (1u << 9), a, b_of(w), 0);
                s.model += 4 * (z.N + 1) + 4ull * z.str_vals[a] + (op == HEDL_OP_SCONTAINS ? 4 * z.contain_words : 0);
                s.n_data++;
            } else {   // role restriction
                const uint32_t c = (uint32_t)sc.k0[i], inv = inv_of(w), a = a_of(w);
                const bool atom = op_of(progs[c]) == HEDL_OP_ATOM && !sc.mat[c];
                const uint32_t ref = atom ? a_of(progs[c]) : (REF_SLOT | read(c));
                if (atom) s.model += z.B;   // the filler concept's row
                put(D_ROLE | (inv << 8) | (op << 16), a, is_count(op) ? b_of(w) : 0u, ref);
                if (s.key == NO_FILLER) s.key = a * 2 + inv;
                if (s.filler == NO_FILLER) s.filler = ref | (op == HEDL_OP_FORALL ? REF_NEG : 0u);
                s.model += 4 * (z.N + 1) + 4ull * z.csr_edges[2 * a + inv] + 2 * z.B;
                s.n_role++;
            }
            depth++;
            if (depth > s.max_depth) s.max_depth = depth;
            fp--;
            continue;
        }
        uint8_t &st = sc.state[o0 + fp - 1];
        if (op == HEDL_OP_NOT) {
            if (st == 0) {
                st = 1;
                sc.stk[o0 + fp] = (uint32_t)sc.k0[i];
                sc.state[o0 + fp] = 0;
                fp++;
            } else {
                put(D_NOT, 0, 0, 0);
                fp--;
            }
            continue;
        }
        // AND / OR: the operand with the larger stack need first
        const int32_t x = sc.k0[i], y = sc.k1[i];
        const uint32_t nx = sc.mat[x] ? 1u : sc.need[x], ny = sc.mat[y] ? 1u : sc.need[y];
        const uint32_t first = (uint32_t)(nx >= ny ? x : y), second = (uint32_t)(nx >= ny ? y : x);
        if (st == 0) {
            st = 1;
            sc.stk[o0 + fp] = first;
            sc.state[o0 + fp] = 0;
            fp++;
        } else if (st == 1) {
            st = 2;
            sc.stk[o0 + fp] = second;
            sc.state[o0 + fp] = 0;
            fp++;
        } else {
            put(op, 0, 0, 0);
            depth--;
            fp--;
        }
    }
    if (reads)   // ascending slot ids (insertion sort: a segment reads few)
        for (uint32_t q = 1; q < s.n_reads; ++q)
            for (uint32_t r = q; r > 0 && reads[r - 1] > reads[r]; --r) {
                const uint32_t t = reads[r];
                reads[r] = reads[r - 1];
                reads[r - 1] = t;
            }
    return s;
}

// ---------------------------------------------------------------- the steps
// The whole pipeline as functions of one index (a hypothesis, a segment, a
// sort position) or of none (the sequential steps), over one context of plain
// pointers: the host driver below runs them in loops (the per-hypothesis ones
// on threads), a device driver runs them as grid-stride kernels.

struct HypCount {           // per hypothesis; scanned in place into offsets
    uint32_t root, n_mat, mat_code, mat_reads, root_code, root_reads, err;
    uint32_t n_role, n_data, n_atom, max_depth;
    uint64_t model;
};

struct Totals {
    uint64_t n_slots, code_n, deps_n, NS, n_levels, WW, TW, n_tiles, n_groups, items;
    uint64_t off_segs, off_deps, off_code, off_ctr, ctr_words;   // set by finish_step
    uint32_t err_hyp, err_code;   // first failing hypothesis (or ERR_BATCH) and its positive error code
};

// err_hyp of a failure of the batch as a whole rather than of one program.
constexpr uint32_t ERR_BATCH = 0xFFFFFFFEu;
// A sort key packs (level, role key, segment) into 14 + 18 + 32 bits, so a
// plan may have at most 2^14 dependency levels (a chain of 16,384 nested role
// restrictions); a deeper batch is refused rather than mis-sorted.
constexpr uint64_t MAX_KEY_LEVELS = 1ull << 14;

// Offsets of the image's tables, as the host planner lays them out (each
// table 256-byte aligned after the header).
struct Layout {
    uint64_t off_segs, off_groups, off_gsegs, off_deps, off_code, off_li, off_ctr, off_slots, off_ft, ctr_words;
};

__host__ __device__ inline uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

__host__ __device__ inline Layout layout(uint64_t NS, uint64_t G, uint64_t D, uint64_t C, uint64_t L, uint64_t H,
                                         uint64_t n_slots, uint64_t B) {
    Layout o{};
    o.off_segs = align256(sizeof(PlanHeader));
    o.off_groups = align256(o.off_segs + NS * sizeof(Seg));
    o.off_gsegs = align256(o.off_groups + G * sizeof(Group));
    o.off_deps = align256(o.off_gsegs + NS * 4);
    o.off_code = align256(o.off_deps + D * 4);
    o.off_li = align256(o.off_code + C * sizeof(DInsn));
    o.off_ctr = align256(o.off_li + (L + 1) * 4);
    o.ctr_words = 4 + (NS + 1) + 2 * H;
    o.off_slots = align256(o.off_ctr + o.ctr_words * 4);   // the (empty) role-group table starts here too
    o.off_ft = align256(o.off_slots + n_slots * B);
    return o;
}

struct Ctx {
    const uint64_t *progs;
    const uint32_t *offs;
    uint32_t H;
    uint32_t n_concepts, n_roles, n_data, n_str, n_patterns;   // id limits (validation)
    bool staged;
    bool validated;            // programs already validated (skip it in count_step)
    Sizes z;
    Scratch sc;
    HypCount *cnt;
    Totals *tot;
    Seg *segs;                 // per segment, in segment order
    DInsn *code;
    uint32_t *deps;
    uint32_t *seg_level, *seg_key;
    uint8_t *seg_walks;
    uint64_t *keys;            // (level, role key, segment), padded with ~0
    uint8_t *starts;           // sorted position starts a group
    uint32_t *segs_at, *walks_at;   // per level
    uint32_t warps, wpl, rounds, timeout_ms, wp, n_sms;
    unsigned flags;
    uint8_t *img;              // the image (zero-filled beforehand)
    uint32_t *level_items;     // [n_levels + 1]
};

// A program's validity as the host planner decides it: HEDL_OK or a negative status.
__host__ __device__ inline int validate(const Ctx &c, uint32_t o0, uint32_t o1) {
    if (o1 <= o0) return HEDL_ERR_BAD_PROGRAM;
    int depth = 0;
    for (uint32_t k = o0; k < o1; ++k) {
        const uint64_t w = c.progs[k];
        const uint32_t op = op_of(w), a = a_of(w);
        if (op < HEDL_OP_ATOM || op > HEDL_OP_SCONTAINS) return HEDL_ERR_BAD_PROGRAM;
        if ((op == HEDL_OP_ATOM && a >= c.n_concepts) || (is_role(op) && a >= c.n_roles) ||
            (is_data(op) && a >= c.n_data) || (is_str(op) && a >= c.n_str) ||
            (op == HEDL_OP_SCONTAINS && b_of(w) >= c.n_patterns))
            return HEDL_ERR_BAD_PROGRAM;
        const int ar = arity(op);
        if (depth < ar) return HEDL_ERR_BAD_PROGRAM;
        depth = depth - ar + 1;
        if (depth > HEDL_MAX_STACK) return HEDL_ERR_BAD_PROGRAM;
    }
    return depth == 1 ? HEDL_OK : HEDL_ERR_BAD_PROGRAM;
}

// Per hypothesis: validate, analyze, count its segments' code and reads.
__host__ __device__ inline void count_step(const Ctx &c, uint32_t h) {
    const uint32_t o0 = c.offs[h], o1 = c.offs[h + 1];
    HypCount &n = c.cnt[h];
    n = HypCount{};
    const int e = o1 < o0 ? HEDL_ERR_INVALID_ARG : (c.validated ? HEDL_OK : validate(c, o0, o1));
    n.err = (uint32_t)-e;
    if (e) return;
    n.root = analyze(c.progs, o0, o1, c.sc, c.staged);
    for (uint32_t k = o0; k < o1; ++k)
        if (c.sc.mat[k]) {
            c.sc.slot[k] = n.n_mat++;
            const SegInfo s = emit(c.progs, o0, c.sc, k, c.z, 0, nullptr, nullptr);
            c.sc.level[k] = s.level;   // operand segments come first: node order
            n.mat_code += s.code_len;
            n.mat_reads += s.n_reads;
        }
    const SegInfo r = emit(c.progs, o0, c.sc, n.root, c.z, 0, nullptr, nullptr);
    n.root_code = r.code_len;
    n.root_reads = r.n_reads;
}

// Sequential: offsets in place (materialised segments of every hypothesis
// first, then the roots), the totals and the first failing hypothesis.
__host__ __device__ inline void scan_step(const Ctx &c) {
    uint64_t slots = 0, code = 0, deps = 0;
    uint32_t err_h = 0xFFFFFFFFu, err_c = 0;
    for (uint32_t h = 0; h < c.H; ++h) {
        HypCount &n = c.cnt[h];
        if (n.err && err_h == 0xFFFFFFFFu) err_h = h, err_c = n.err;
        const uint32_t m = n.n_mat, mc = n.mat_code, md = n.mat_reads;
        n.n_mat = (uint32_t)slots;
        n.mat_code = (uint32_t)code;
        n.mat_reads = (uint32_t)deps;
        slots += m;
        code += mc;
        deps += md;
    }
    for (uint32_t h = 0; h < c.H; ++h) {
        HypCount &n = c.cnt[h];
        const uint32_t rc = n.root_code, rd = n.root_reads;
        n.root_code = (uint32_t)code;
        n.root_reads = (uint32_t)deps;
        code += rc;
        deps += rd;
    }
    Totals &t = *c.tot;
    t = Totals{};
    t.n_slots = slots;
    t.code_n = code;
    t.deps_n = deps;
    t.NS = slots + c.H;
    t.err_hyp = err_h;
    t.err_code = err_c;
}

// Per hypothesis: emit its segments at their offsets.
__host__ __device__ inline void write_step(const Ctx &c, uint32_t h) {
    if (c.tot->err_hyp != 0xFFFFFFFFu) return;
    const uint32_t o0 = c.offs[h], o1 = c.offs[h + 1];
    HypCount &n = c.cnt[h];
    const uint32_t slot_base = n.n_mat;
    uint32_t c_at = n.mat_code, d_at = n.mat_reads;
    auto record = [&](uint32_t sidx, const SegInfo &s, uint32_t c0, uint32_t d0, uint32_t out_slot, uint32_t hyp) {
        Seg g{};
        g.code_off = c0;
        g.code_len = s.code_len;
        g.out_slot = out_slot;
        g.hyp = hyp;
        g.dep_off = d0;
        g.dep_cnt = s.n_reads;
        g.filler = s.filler;
        g.kind = TASK_SEGMENT;
        c.segs[sidx] = g;
        c.seg_level[sidx] = s.level;
        c.seg_key[sidx] = s.key;
        c.seg_walks[sidx] = s.key != NO_FILLER;
        n.model += s.model;
        n.n_role += s.n_role;
        n.n_data += s.n_data;
        n.n_atom += s.n_atom;
        if (s.max_depth > n.max_depth) n.max_depth = s.max_depth;
    };
    for (uint32_t k = o0; k < o1; ++k)
        if (c.sc.mat[k]) {
            const SegInfo s = emit(c.progs, o0, c.sc, k, c.z, slot_base, c.code + c_at, c.deps + d_at);
            c.sc.level[k] = s.level;
            record(slot_base + c.sc.slot[k], s, c_at, d_at, slot_base + c.sc.slot[k], NO_HYP);
            c_at += s.code_len;
            d_at += s.n_reads;
        }
    const SegInfo r = emit(c.progs, o0, c.sc, n.root, c.z, slot_base, c.code + n.root_code, c.deps + n.root_reads);
    record((uint32_t)c.tot->n_slots + h, r, n.root_code, n.root_reads, NO_SLOT, h);
    n.model += 2 * c.z.B + 16;   // the hypothesis's score
}

// Sequential: levels, and the tile shape by the host planner's rule (a warp
// covers fewer words when a level that walks a role has few segments).
__host__ __device__ inline void shape_step(const Ctx &c) {
    Totals &t = *c.tot;
    if (t.err_hyp != 0xFFFFFFFFu) return;
    uint32_t n_levels = 0;
    for (uint64_t s = 0; s < t.NS; ++s) n_levels = c.seg_level[s] + 1 > n_levels ? c.seg_level[s] + 1 : n_levels;
    if (n_levels > MAX_KEY_LEVELS) {
        t.err_hyp = ERR_BATCH;
        t.err_code = (uint32_t)-HEDL_ERR_INVALID_ARG;
        return;
    }
    for (uint32_t L = 0; L < n_levels; ++L) c.segs_at[L] = c.walks_at[L] = 0;
    for (uint64_t s = 0; s < t.NS; ++s) {
        c.segs_at[c.seg_level[s]]++;
        c.walks_at[c.seg_level[s]] |= c.seg_walks[s];
    }
    uint64_t smin = ~0ull;
    for (uint32_t L = 0; L < n_levels; ++L)
        if (c.walks_at[L] && c.segs_at[L] < smin) smin = c.segs_at[L];
    uint32_t WW = 32, rounds = c.rounds;
    if (c.n_sms > 0) {
        const uint64_t resident = 32ull * c.n_sms;
        if (smin != ~0ull)
            while (WW > 4 && smin * c.wp < 4ull * resident * WW * c.wpl) WW >>= 1;
        if (WW < 32) rounds = 1;
    }
    t.n_levels = n_levels;
    t.WW = WW;
    t.TW = (uint64_t)c.warps * WW * c.wpl * rounds;
    t.n_tiles = (c.wp + t.TW - 1) / t.TW;
}

// Per sort position: the key of segment i (unique, so any sort is the stable one).
__host__ __device__ inline void key_step(const Ctx &c, uint64_t i) {
    if (i < c.tot->NS) {
        const uint64_t key = c.seg_key[i] == NO_FILLER ? (1ull << 17) : (uint64_t)c.seg_key[i];   // role keys < 2^17
        c.keys[i] = ((uint64_t)c.seg_level[i] << 50) | (key << 32) | i;
    } else {
        c.keys[i] = ~0ull;
    }
}

// Per sort position: one compare-exchange of a bitonic step (n2 a power of two).
__host__ __device__ inline void bitonic_step(uint64_t *keys, uint64_t i, uint64_t j, uint64_t k) {
    const uint64_t l = i ^ j;
    if (l > i) {
        const uint64_t a = keys[i], b = keys[l];
        if ((a > b) == ((i & k) == 0)) {
            keys[i] = b;
            keys[l] = a;
        }
    }
}

// Per sorted position: does it start a group (a new (level, role key))?
__host__ __device__ inline void start_step(const Ctx &c, uint64_t i) {
    if (i < c.tot->NS) c.starts[i] = i == 0 || (c.keys[i] >> 32) != (c.keys[i - 1] >> 32);
}

// The header and the totals of a plan with G groups, once the groups, gsegs
// and level items are in the image (both drivers).
__host__ __device__ inline void header_step(const Ctx &c, uint64_t G) {
    Totals &t = *c.tot;
    const uint64_t NS = t.NS, n_tiles = t.n_tiles, L = t.n_levels;
    const Layout o = layout(NS, G, t.deps_n, t.code_n, L, c.H, t.n_slots, c.z.B);
    PlanHeader hd{};
    hd.n_items = (uint32_t)(NS * n_tiles);
    hd.n_segs = (uint32_t)NS;
    hd.n_groups = (uint32_t)G;
    hd.n_hyps = c.H;
    hd.n_tiles = (uint32_t)n_tiles;
    hd.tile_words = (uint32_t)t.TW;
    hd.n_slots = (uint32_t)t.n_slots;
    hd.flags = c.flags;
    hd.n_levels = (uint32_t)L;
    hd.n_deps = (uint32_t)t.deps_n;
    hd.n_rgroups = 0;
    hd.warp_words = (uint32_t)t.WW;
    hd.off_segs = o.off_segs;
    hd.off_groups = o.off_groups;
    hd.off_gsegs = o.off_gsegs;
    hd.off_deps = o.off_deps;
    hd.off_code = o.off_code;
    hd.off_level_items = o.off_li;
    hd.off_ctr = o.off_ctr;
    hd.off_slots = o.off_slots;
    hd.off_rgroups = o.off_slots;
    hd.off_ft = o.off_ft;
    hd.timeout_ns = (uint64_t)c.timeout_ms * 1000000ull;
    *reinterpret_cast<PlanHeader *>(c.img) = hd;
    t.n_groups = G;
    t.items = NS * n_tiles;
    t.off_segs = o.off_segs;
    t.off_deps = o.off_deps;
    t.off_code = o.off_code;
    t.off_ctr = o.off_ctr;
    t.ctr_words = o.ctr_words;
}

// Sequential: groups, gsegs, level_items and the header.
__host__ __device__ inline void finish_step(const Ctx &c) {
    Totals &t = *c.tot;
    if (t.err_hyp != 0xFFFFFFFFu) return;
    const uint64_t NS = t.NS, n_tiles = t.n_tiles, L = t.n_levels;
    uint64_t G = 0;
    for (uint64_t i = 0; i < NS; ++i) G += c.starts[i];
    const Layout o = layout(NS, G, t.deps_n, t.code_n, L, c.H, t.n_slots, c.z.B);
    Group *groups = reinterpret_cast<Group *>(c.img + o.off_groups);
    uint32_t *gsegs = reinterpret_cast<uint32_t *>(c.img + o.off_gsegs);
    uint32_t *li = reinterpret_cast<uint32_t *>(c.img + o.off_li);
    for (uint64_t l = 0; l <= L; ++l) li[l] = 0;
    uint64_t g = 0, begin = 0;
    for (uint64_t i = 0; i < NS; ++i) {
        gsegs[i] = (uint32_t)(c.keys[i] & 0xFFFFFFFFull);
        if (c.starts[i]) begin = i;
        if (i + 1 == NS || c.starts[i + 1]) {   // the group [begin, i] ends here
            const uint32_t lvl = c.seg_level[gsegs[begin]];
            groups[g++] = Group{(uint32_t)(begin * n_tiles), (uint32_t)begin, (uint32_t)(i + 1 - begin), lvl};
            li[lvl + 1] = (uint32_t)((i + 1) * n_tiles);
        }
    }
    for (uint64_t l = 1; l <= L; ++l) li[l] = li[l] > li[l - 1] ? li[l] : li[l - 1];
    for (uint64_t l = 0; l <= L; ++l) c.level_items[l] = li[l];
    header_step(c, G);
}

// Per index: copy segment i, dependency i and code word i into the image; zero counter i.
__host__ __device__ inline void assemble_step(const Ctx &c, uint64_t i) {
    const Totals &t = *c.tot;
    if (t.err_hyp != 0xFFFFFFFFu) return;
    if (i < t.NS) reinterpret_cast<Seg *>(c.img + t.off_segs)[i] = c.segs[i];
    if (i < t.deps_n) reinterpret_cast<uint32_t *>(c.img + t.off_deps)[i] = c.deps[i];
    if (i < t.code_n) reinterpret_cast<DInsn *>(c.img + t.off_code)[i] = c.code[i];
    if (i < t.ctr_words) reinterpret_cast<uint32_t *>(c.img + t.off_ctr)[i] = 0;
}

// Upper bounds from the instruction count NI and H, known before planning.
struct Bounds {
    uint64_t NS, code, deps, levels, slots;
};
__host__ __device__ inline Bounds bounds(uint64_t NI, uint64_t H) { return Bounds{NI + H, 2 * NI, NI, NI + 1, NI}; }

__host__ __device__ inline uint64_t pow2_at_least(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// ---------------------------------------------------------------- the device driver's kernels
// The per-index steps above as grid-stride kernels; the sequential steps as
// one-block kernels built on block-wide scans and reductions.

constexpr int SCAN_THREADS = 1024;

__device__ inline uint64_t gstride() { return (uint64_t)gridDim.x * blockDim.x; }
__device__ inline uint64_t gindex() { return (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; }

// Inclusive scan of one value per thread over a block of SCAN_THREADS threads.
__device__ inline uint64_t block_inclusive_scan(uint64_t x, uint64_t *sh) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < (blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= (uint32_t)o) w += y;
        }
        sh[lane] = w;
    }
    __syncthreads();
    const uint64_t r = x + (warp ? sh[warp - 1] : 0);
    __syncthreads();
    return r;
}

// Per hypothesis: offsets bounds first (a program outside [0, n_insns) is
// refused before any scratch is touched), then count_step.
__global__ void count_kernel(Ctx c, uint64_t n_insns) {
    for (uint64_t h = gindex(); h < c.H; h += gstride()) {
        const uint32_t o0 = c.offs[h], o1 = c.offs[h + 1];
        if ((h == 0 && o0 != 0) || o1 < o0 || o1 > n_insns || (h + 1 == c.H && o1 != n_insns)) {
            c.cnt[h] = HypCount{};
            c.cnt[h].err = (uint32_t)-HEDL_ERR_INVALID_ARG;
            continue;
        }
        count_step(c, (uint32_t)h);
    }
}

// scan_step's offsets and totals by block-wide scans (one block of SCAN_THREADS):
// each thread sums a contiguous stretch of hypotheses, the block scans the
// stretch sums, and each thread writes its stretch's offsets.
__global__ void __launch_bounds__(SCAN_THREADS) scan_kernel(Ctx c) {
    __shared__ uint64_t sh[32];
    __shared__ uint64_t tot_mat_code, tot_mat_reads;
    __shared__ uint32_t first_err;
    const uint32_t T = blockDim.x, t = threadIdx.x;
    const uint32_t per = (c.H + T - 1) / T;
    const uint32_t h0 = min(c.H, t * per), h1 = min(c.H, h0 + per);
    if (t == 0) first_err = 0xFFFFFFFFu;
    __syncthreads();
    uint64_t slots = 0, code = 0, deps = 0, rcode = 0, rdeps = 0;
    for (uint32_t h = h0; h < h1; ++h) {
        const HypCount &n = c.cnt[h];
        if (n.err) atomicMin(&first_err, h);
        slots += n.n_mat;
        code += n.mat_code;
        deps += n.mat_reads;
        rcode += n.root_code;
        rdeps += n.root_reads;
    }
    const uint64_t i_slots = block_inclusive_scan(slots, sh), i_code = block_inclusive_scan(code, sh);
    const uint64_t i_deps = block_inclusive_scan(deps, sh), i_rcode = block_inclusive_scan(rcode, sh);
    const uint64_t i_rdeps = block_inclusive_scan(rdeps, sh);
    if (t == T - 1) {
        tot_mat_code = i_code;
        tot_mat_reads = i_deps;
    }
    __syncthreads();
    uint64_t a_slots = i_slots - slots, a_code = i_code - code, a_deps = i_deps - deps;
    uint64_t a_rcode = tot_mat_code + i_rcode - rcode, a_rdeps = tot_mat_reads + i_rdeps - rdeps;
    for (uint32_t h = h0; h < h1; ++h) {
        HypCount &n = c.cnt[h];
        const uint32_t m = n.n_mat, mc = n.mat_code, md = n.mat_reads, rc = n.root_code, rd = n.root_reads;
        n.n_mat = (uint32_t)a_slots;
        n.mat_code = (uint32_t)a_code;
        n.mat_reads = (uint32_t)a_deps;
        n.root_code = (uint32_t)a_rcode;
        n.root_reads = (uint32_t)a_rdeps;
        a_slots += m;
        a_code += mc;
        a_deps += md;
        a_rcode += rc;
        a_rdeps += rd;
    }
    if (t == T - 1) {
        Totals &tt = *c.tot;
        tt = Totals{};
        tt.n_slots = i_slots;
        tt.code_n = tot_mat_code + i_rcode;
        tt.deps_n = tot_mat_reads + i_rdeps;
        tt.NS = i_slots + c.H;
        tt.err_hyp = first_err;
        tt.err_code = first_err == 0xFFFFFFFFu ? 0u : c.cnt[first_err].err;
    }
}

__global__ void write_kernel(Ctx c) {
    for (uint64_t h = gindex(); h < c.H; h += gstride()) write_step(c, (uint32_t)h);
}

// shape_step by block-wide reductions (one block): the level count, the
// segments (and role-walking segments) per level, the narrowest level, then
// the tile shape by thread 0.
__global__ void __launch_bounds__(SCAN_THREADS) shape_kernel(Ctx c) {
    Totals &t = *c.tot;
    if (t.err_hyp != 0xFFFFFFFFu) return;
    __shared__ uint32_t n_levels;
    __shared__ unsigned long long smin;
    if (threadIdx.x == 0) {
        n_levels = 0;
        smin = ~0ull;
    }
    __syncthreads();
    for (uint64_t s = threadIdx.x; s < t.NS; s += blockDim.x) atomicMax(&n_levels, c.seg_level[s] + 1);
    __syncthreads();
    const uint32_t L = n_levels;
    if ((uint64_t)L > MAX_KEY_LEVELS) {
        if (threadIdx.x == 0) {
            t.err_hyp = ERR_BATCH;
            t.err_code = (uint32_t)-HEDL_ERR_INVALID_ARG;
        }
        return;
    }
    for (uint32_t l = threadIdx.x; l < L; l += blockDim.x) c.segs_at[l] = c.walks_at[l] = 0;
    __syncthreads();
    for (uint64_t s = threadIdx.x; s < t.NS; s += blockDim.x) {
        atomicAdd(&c.segs_at[c.seg_level[s]], 1u);
        if (c.seg_walks[s]) atomicOr(&c.walks_at[c.seg_level[s]], 1u);
    }
    __threadfence_block();
    __syncthreads();
    for (uint32_t l = threadIdx.x; l < L; l += blockDim.x)
        if (__ldcg(c.walks_at + l)) atomicMin(&smin, (unsigned long long)__ldcg(c.segs_at + l));
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t WW = 32, rounds = c.rounds;
        if (c.n_sms > 0) {
            const uint64_t resident = 32ull * c.n_sms;
            if (smin != ~0ull)
                while (WW > 4 && smin * c.wp < 4ull * resident * WW * c.wpl) WW >>= 1;
            if (WW < 32) rounds = 1;
        }
        t.n_levels = L;
        t.WW = WW;
        t.TW = (uint64_t)c.warps * WW * c.wpl * rounds;
        t.n_tiles = (c.wp + t.TW - 1) / t.TW;
    }
}

__global__ void key_kernel(Ctx c, uint64_t n2) {
    if (c.tot->err_hyp != 0xFFFFFFFFu) return;
    for (uint64_t i = gindex(); i < n2; i += gstride()) key_step(c, i);
}

// One compare-exchange step (j, k) of the bitonic network over all n2 keys.
__global__ void bitonic_global_kernel(uint64_t *keys, uint64_t n2, uint64_t j, uint64_t k) {
    for (uint64_t i = gindex(); i < n2; i += gstride()) bitonic_step(keys, i, j, k);
}

constexpr uint32_t BITONIC_TILE = 2048;   // keys a block sorts in shared memory (16 KB)

// The steps of the network whose partners lie within one tile of BITONIC_TILE
// keys: every k from k_from to k_to (powers of two), each with j from
// min(j_from, k / 2) down to 1; a block holds one tile in shared memory.
__global__ void __launch_bounds__(1024) bitonic_tile_kernel(uint64_t *keys, uint64_t n2, uint64_t k_from,
                                                            uint64_t k_to, uint64_t j_from) {
    __shared__ uint64_t sk[BITONIC_TILE];
    const uint64_t base = (uint64_t)blockIdx.x * BITONIC_TILE;
    const uint32_t span = (uint32_t)(n2 - base < BITONIC_TILE ? n2 - base : (uint64_t)BITONIC_TILE);
    for (uint32_t q = threadIdx.x; q < span; q += blockDim.x) sk[q] = keys[base + q];
    __syncthreads();
    for (uint64_t k = k_from; k <= k_to; k <<= 1) {
        for (uint64_t j = (j_from < (k >> 1) ? j_from : (k >> 1)); j > 0; j >>= 1) {
            for (uint32_t q = threadIdx.x; q < span; q += blockDim.x) {
                const uint64_t i = base + q, l = i ^ j;   // l stays inside the tile: j < BITONIC_TILE
                if (l > i) {
                    const uint64_t a = sk[q], b = sk[l - base];
                    if ((a > b) == ((i & k) == 0)) {
                        sk[q] = b;
                        sk[l - base] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t q = threadIdx.x; q < span; q += blockDim.x) keys[base + q] = sk[q];
}

__global__ void start_kernel(Ctx c) {
    if (c.tot->err_hyp != 0xFFFFFFFFu) return;
    for (uint64_t i = gindex(); i < c.tot->NS; i += gstride()) start_step(c, i);
}

// Group index of every sorted position (exclusive scan of the starts, one
// block), the group count, and the zeroed level items.
__global__ void __launch_bounds__(SCAN_THREADS) group_scan_kernel(Ctx c, uint32_t *gidx, uint64_t *G_out) {
    Totals &t = *c.tot;
    if (t.err_hyp != 0xFFFFFFFFu) return;
    __shared__ uint64_t sh[32];
    const uint64_t NS = t.NS, T = blockDim.x, per = (NS + T - 1) / T;
    const uint64_t i0 = min(NS, threadIdx.x * per), i1 = min(NS, i0 + per);
    uint64_t cnt = 0;
    for (uint64_t i = i0; i < i1; ++i) cnt += c.starts[i];
    const uint64_t incl = block_inclusive_scan(cnt, sh);
    uint64_t g = incl - cnt;
    for (uint64_t i = i0; i < i1; ++i) {
        g += c.starts[i];
        gidx[i] = (uint32_t)(g - 1);   // the group position i belongs to
    }
    if (threadIdx.x == T - 1) *G_out = incl;
}

// Per sorted position: gsegs, and the group that ends there (with its first
// position found by the group's start), and its level's item bound.
__global__ void group_kernel(Ctx c, const uint32_t *gidx, const uint64_t *G_in, uint64_t *gbegin) {
    Totals &t = *c.tot;
    if (t.err_hyp != 0xFFFFFFFFu) return;
    const uint64_t NS = t.NS, n_tiles = t.n_tiles;
    const Layout o = layout(NS, *G_in, t.deps_n, t.code_n, t.n_levels, c.H, t.n_slots, c.z.B);
    uint32_t *gsegs = reinterpret_cast<uint32_t *>(c.img + o.off_gsegs);
    for (uint64_t i = gindex(); i < NS; i += gstride()) {
        gsegs[i] = (uint32_t)(c.keys[i] & 0xFFFFFFFFull);
        if (c.starts[i]) gbegin[gidx[i]] = i;
    }
}

__global__ void group_end_kernel(Ctx c, const uint32_t *gidx, const uint64_t *G_in, const uint64_t *gbegin) {
    Totals &t = *c.tot;
    if (t.err_hyp != 0xFFFFFFFFu) return;
    const uint64_t NS = t.NS, n_tiles = t.n_tiles;
    const Layout o = layout(NS, *G_in, t.deps_n, t.code_n, t.n_levels, c.H, t.n_slots, c.z.B);
    Group *groups = reinterpret_cast<Group *>(c.img + o.off_groups);
    uint32_t *li = reinterpret_cast<uint32_t *>(c.img + o.off_li);
    for (uint64_t i = gindex(); i < NS; i += gstride()) {
        if (i + 1 == NS || c.starts[i + 1]) {
            const uint64_t g = gidx[i], begin = gbegin[g];
            const uint32_t lvl = c.seg_level[(uint32_t)(c.keys[begin] & 0xFFFFFFFFull)];
            groups[g] = Group{(uint32_t)(begin * n_tiles), (uint32_t)begin, (uint32_t)(i + 1 - begin), lvl};
            atomicMax(li + lvl + 1, (uint32_t)((i + 1) * n_tiles));
        }
    }
}

// The level items' running maximum (levels in order), then the header.
__global__ void header_kernel(Ctx c, const uint64_t *G_in) {
    Totals &t = *c.tot;
    if (t.err_hyp != 0xFFFFFFFFu) return;
    const uint64_t L = t.n_levels;
    const Layout o = layout(t.NS, *G_in, t.deps_n, t.code_n, L, c.H, t.n_slots, c.z.B);
    uint32_t *li = reinterpret_cast<uint32_t *>(c.img + o.off_li);
    for (uint64_t l = 1; l <= L; ++l) li[l] = li[l] > li[l - 1] ? li[l] : li[l - 1];
    for (uint64_t l = 0; l <= L; ++l) c.level_items[l] = li[l];
    header_step(c, *G_in);
}

__global__ void assemble_kernel(Ctx c, uint64_t span) {
    if (c.tot->err_hyp != 0xFFFFFFFFu) return;
    for (uint64_t i = gindex(); i < span; i += gstride()) assemble_step(c, i);
}

}  // namespace dp

namespace {

// Run f(h) for h in [0, H) on n threads (contiguous shares).
template <typename F>
void parallel_for(uint32_t H, uint32_t n, F f) {
    n = std::max<uint32_t>(1, std::min<uint32_t>(n, H));
    if (n == 1) {
        for (uint32_t h = 0; h < H; ++h) f(h);
        return;
    }
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < n; ++t)
        th.emplace_back([=, &f] {
            for (uint32_t h = (uint32_t)((uint64_t)H * t / n); h < (uint32_t)((uint64_t)H * (t + 1) / n); ++h) f(h);
        });
    for (auto &x : th) x.join();
}

}  // namespace

int build_plan_parallel(const hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, unsigned flags,
                        uint32_t n_threads, PlanImpl **out) {
    *out = nullptr;
    if (H == 0) return fail(HEDL_ERR_INVALID_ARG, "empty batch (H = 0)");
    if (flags & (HEDL_PLAIN | HEDL_TEST_UNSAT_DEP | HEDL_SLICE_ALL))
        return fail(HEDL_ERR_INVALID_ARG, "the parallel planner takes neither HEDL_PLAIN, HEDL_SLICE_ALL nor test flags");
    for (uint32_t h = 0; h < H; ++h)
        if (offs[h + 1] < offs[h]) return fail(HEDL_ERR_INVALID_ARG, "offs must be non-decreasing");
    flags |= HEDL_NO_CSE | HEDL_NO_SLICE;
    if (!n_threads) n_threads = std::max(1u, std::thread::hardware_concurrency());
    {   // validation with messages, per hypothesis in parallel; the first bad program is reported
        std::vector<int> err(H, 0);
        std::vector<std::string> why(H);
        parallel_for(H, n_threads, [&](uint32_t h) {
            err[h] = validate_program(kb, progs + offs[h], offs[h + 1] - offs[h], &why[h]);
        });
        for (uint32_t h = 0; h < H; ++h)
            if (err[h]) return fail(err[h], "program " + std::to_string(h) + ": " + why[h]);
    }
    const uint64_t NI = offs[H];
    const dp::Bounds b = dp::bounds(NI, H);
    std::vector<uint32_t> num_vals, str_vals, csr_edges;
    for (const DevNum &g : kb->num_host) num_vals.push_back(g.n_vals);
    for (const DevStr &g : kb->str_host) str_vals.push_back(g.n_vals);
    for (const DevCSR &g : kb->csr_host) csr_edges.push_back(g.n_edges);
    // scratch: every entry is written before it is read, so it is left uninitialised
    auto buf = [](uint64_t n, auto *tag) { return std::unique_ptr<std::remove_pointer_t<decltype(tag)>[]>(
                                               new std::remove_pointer_t<decltype(tag)>[n ? n : 1]); };
    auto k0 = buf(NI, (int32_t *)nullptr), k1 = buf(NI, (int32_t *)nullptr);
    auto need = buf(NI, (uint32_t *)nullptr), slot = buf(NI, (uint32_t *)nullptr);
    auto level = buf(NI, (uint32_t *)nullptr), stk = buf(NI, (uint32_t *)nullptr);
    auto mat = buf(NI, (uint8_t *)nullptr), state = buf(NI, (uint8_t *)nullptr);
    std::vector<dp::HypCount> cnt(H);
    dp::Totals tot{};
    auto segs = buf(b.NS, (Seg *)nullptr);
    auto code = buf(b.code, (DInsn *)nullptr);
    auto deps = buf(b.deps, (uint32_t *)nullptr);
    auto seg_level = buf(b.NS, (uint32_t *)nullptr), seg_key = buf(b.NS, (uint32_t *)nullptr);
    auto seg_walks = buf(b.NS, (uint8_t *)nullptr), starts = buf(b.NS, (uint8_t *)nullptr);
    auto keys = buf(b.NS, (uint64_t *)nullptr);
    std::vector<uint32_t> segs_at(b.levels), walks_at(b.levels), level_items(b.levels + 1);
    std::vector<uint8_t> img;   // sized once the groups are known

    dp::Ctx c{};
    c.progs = progs;
    c.offs = offs;
    c.H = H;
    c.n_concepts = kb->n_concepts;
    c.n_roles = kb->n_roles;
    c.n_data = kb->n_props + kb->n_num;
    c.n_str = kb->n_str;
    c.n_patterns = kb->n_patterns;
    c.staged = use_staging(kb, kb->tuning);
    c.validated = true;
    c.z = dp::Sizes{kb->n, 4ull * kb->wp, kb->n_props, num_vals.data(), str_vals.data(), csr_edges.data(),
                    kb->contain_words};
    c.sc = dp::Scratch{k0.get(), k1.get(), need.get(), mat.get(), slot.get(), level.get(), stk.get(), state.get()};
    c.cnt = cnt.data();
    c.tot = &tot;
    c.segs = segs.get();
    c.code = code.get();
    c.deps = deps.get();
    c.seg_level = seg_level.get();
    c.seg_key = seg_key.get();
    c.seg_walks = seg_walks.get();
    c.keys = keys.get();
    c.starts = starts.get();
    c.segs_at = segs_at.data();
    c.walks_at = walks_at.data();
    const Tuning &tu = kb->tuning;
    c.warps = tu.warps;
    c.wpl = tu.wpl;
    c.rounds = tu.rounds;
    c.timeout_ms = tu.timeout_ms;
    c.wp = kb->wp;
    c.n_sms = (uint32_t)std::max(kb->n_sms, 0);
    c.flags = flags;
    c.level_items = level_items.data();

    // the steps: per hypothesis on threads, the sequential ones in turn; the
    // sort of unique keys is std::sort here (a bitonic network on the device)
    parallel_for(H, n_threads, [&](uint32_t h) { dp::count_step(c, h); });
    dp::scan_step(c);
    if (tot.err_hyp != 0xFFFFFFFFu)
        return fail(-(int)tot.err_code, "program " + std::to_string(tot.err_hyp) + " is not valid");
    if (tot.n_slots > REF_ID) return fail(HEDL_ERR_INVALID_ARG, "batch too large: more than 2^30 materialized intermediate sets");
    parallel_for(H, n_threads, [&](uint32_t h) { dp::write_step(c, h); });
    dp::shape_step(c);
    if (tot.err_hyp == dp::ERR_BATCH)
        return fail(HEDL_ERR_INVALID_ARG, "batch too deep for the per-hypothesis planner: more than 16,384 dependency "
                                          "levels (nested role restrictions); plan it with hedl_plan_batch");
    for (uint64_t i = 0; i < tot.NS; ++i) dp::key_step(c, i);
    std::sort(keys.get(), keys.get() + tot.NS);
    uint64_t G = 0;
    for (uint64_t i = 0; i < tot.NS; ++i) {
        dp::start_step(c, i);
        G += starts[i];
    }
    img.assign(dp::layout(tot.NS, G, tot.deps_n, tot.code_n, tot.n_levels, H, tot.n_slots, 4ull * kb->wp).off_slots, 0);
    c.img = img.data();
    dp::finish_step(c);
    const uint64_t span = std::max<uint64_t>(std::max<uint64_t>(tot.NS, tot.code_n), std::max<uint64_t>(tot.deps_n, 4 + tot.NS + 1 + 2ull * H));
    for (uint64_t i = 0; i < span; ++i) dp::assemble_step(c, i);
    if (tot.items >= 0xFFFFFFFFull) return fail(HEDL_ERR_INVALID_ARG, "batch too large: more than 2^32 work items");

    PlanHeader hd;
    memcpy(&hd, img.data(), sizeof hd);
    auto *p = new PlanImpl();
    p->flags = flags;
    p->n_hyps = H;
    p->tuning = kb->tuning;
    p->staged = c.staged;
    p->info.n_hyps = H;
    p->info.total_insns = NI;
    p->info.n_nodes = NI;
    uint64_t model = 0;
    for (const dp::HypCount &n : cnt) {
        model += n.model;
        p->info.n_role_ops += n.n_role;
        p->info.n_data_ops += n.n_data;
        p->info.n_atom_loads += n.n_atom;
        p->max_stack = std::max(p->max_stack, n.max_depth);
    }
    if (p->max_stack > (uint32_t)STACK_MAX) {
        delete p;
        return fail(HEDL_ERR_BAD_PROGRAM, "internal: segment stack exceeds the device limit");
    }
    p->image = std::move(img);
    p->image_bytes = hd.off_slots;
    p->ctr_off = hd.off_ctr;
    p->ctr_bytes = (4 + (uint64_t)(tot.NS + 1) + 2ull * H) * 4;
    p->slots_off = hd.off_slots;
    p->ws_bytes = hd.off_ft;
    p->n_rgroups = 0;
    p->level_items.assign(level_items.begin(), level_items.begin() + tot.n_levels + 1);
    p->info.n_segments = hd.n_segs;
    p->info.n_slots = hd.n_slots;
    p->info.n_levels = hd.n_levels;
    p->info.n_items = hd.n_items;
    p->info.tile_words = hd.tile_words;
    p->info.warp_words = hd.warp_words;
    p->info.workspace_bytes = p->ws_bytes;
    p->info.image_bytes = p->image_bytes;
    p->info.model_bytes = model;
    *out = p;
    return HEDL_OK;
}

namespace {

// One device allocation carved into 256-byte aligned pieces.
struct Carve {
    uint8_t *base = nullptr;
    uint64_t at = 0;
    template <typename T>
    T *take(uint64_t n) {
        T *p = reinterpret_cast<T *>(base + at);
        at = (at + sizeof(T) * (n ? n : 1) + 255) & ~uint64_t(255);
        return p;
    }
};

uint32_t grid_for(uint64_t n, uint32_t threads) {
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((n + threads - 1) / threads, 4096));
}

}  // namespace

// The device-side planner: the same steps as build_plan_parallel, launched as
// kernels over device programs.  Two host synchronisations: after the scan
// (the totals size the image) and at the end (the header, level items and
// per-hypothesis counts come back for the plan's info).
int build_plan_device(const hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, uint64_t NI,
                      unsigned flags, cudaStream_t st, PlanImpl **out) {
    *out = nullptr;
    if (H == 0) return fail(HEDL_ERR_INVALID_ARG, "empty batch (H = 0)");
    if (kb->plan_only) return fail(HEDL_ERR_INVALID_ARG, "planning-only handle: the device planner needs a GPU");
    if (NI == 0 || NI >= 0xFFFFFFFFull) return fail(HEDL_ERR_INVALID_ARG, "n_insns must be in [1, 2^32 - 1)");
    if (flags & (HEDL_PLAIN | HEDL_TEST_UNSAT_DEP | HEDL_SLICE_ALL))
        return fail(HEDL_ERR_INVALID_ARG, "the device planner takes neither HEDL_PLAIN, HEDL_SLICE_ALL nor test flags");
    flags |= HEDL_NO_CSE | HEDL_NO_SLICE;
    const dp::Bounds b = dp::bounds(NI, H);
    const uint64_t n2max = dp::pow2_at_least(b.NS);
    std::vector<uint32_t> num_vals, str_vals, csr_edges;
    for (const DevNum &g : kb->num_host) num_vals.push_back(g.n_vals);
    for (const DevStr &g : kb->str_host) str_vals.push_back(g.n_vals);
    for (const DevCSR &g : kb->csr_host) csr_edges.push_back(g.n_edges);
    // the scratch, carved once the sizes are summed
    auto carve_all = [&](Carve &cv, dp::Ctx &c, uint32_t **gidx, uint64_t **gbegin, uint64_t **G,
                         uint32_t **dnum, uint32_t **dstr, uint32_t **dcsr) {
        c.sc.k0 = cv.take<int32_t>(NI);
        c.sc.k1 = cv.take<int32_t>(NI);
        c.sc.need = cv.take<uint32_t>(NI);
        c.sc.slot = cv.take<uint32_t>(NI);
        c.sc.level = cv.take<uint32_t>(NI);
        c.sc.stk = cv.take<uint32_t>(NI);
        c.sc.mat = cv.take<uint8_t>(NI);
        c.sc.state = cv.take<uint8_t>(NI);
        c.cnt = cv.take<dp::HypCount>(H);
        c.tot = cv.take<dp::Totals>(1);
        c.segs = cv.take<Seg>(b.NS);
        c.code = cv.take<DInsn>(b.code);
        c.deps = cv.take<uint32_t>(b.deps);
        c.seg_level = cv.take<uint32_t>(b.NS);
        c.seg_key = cv.take<uint32_t>(b.NS);
        c.seg_walks = cv.take<uint8_t>(b.NS);
        c.starts = cv.take<uint8_t>(b.NS);
        c.keys = cv.take<uint64_t>(n2max);
        c.segs_at = cv.take<uint32_t>(b.levels);
        c.walks_at = cv.take<uint32_t>(b.levels);
        c.level_items = cv.take<uint32_t>(b.levels + 1);
        *gidx = cv.take<uint32_t>(b.NS);
        *gbegin = cv.take<uint64_t>(b.NS);
        *G = cv.take<uint64_t>(1);
        *dnum = cv.take<uint32_t>(num_vals.size());
        *dstr = cv.take<uint32_t>(str_vals.size());
        *dcsr = cv.take<uint32_t>(csr_edges.size());
    };
    dp::Ctx c{};
    uint32_t *gidx, *dnum, *dstr, *dcsr;
    uint64_t *gbegin, *Gd;
    Carve sizing;
    carve_all(sizing, c, &gidx, &gbegin, &Gd, &dnum, &dstr, &dcsr);
    void *scratch = nullptr;
    cudaError_t e = cudaMalloc(&scratch, sizing.at);
    if (e) return cuda_fail(e, "device planner scratch");
    std::unique_ptr<void, void (*)(void *)> scratch_guard(scratch, [](void *q) { cudaFree(q); });
    Carve cv;
    cv.base = (uint8_t *)scratch;
    carve_all(cv, c, &gidx, &gbegin, &Gd, &dnum, &dstr, &dcsr);
    if (!num_vals.empty()) e = cudaMemcpyAsync(dnum, num_vals.data(), 4 * num_vals.size(), cudaMemcpyHostToDevice, st);
    if (!e && !str_vals.empty()) e = cudaMemcpyAsync(dstr, str_vals.data(), 4 * str_vals.size(), cudaMemcpyHostToDevice, st);
    if (!e && !csr_edges.empty()) e = cudaMemcpyAsync(dcsr, csr_edges.data(), 4 * csr_edges.size(), cudaMemcpyHostToDevice, st);
    if (e) return cuda_fail(e, "device planner sizes");
    c.progs = progs;
    c.offs = offs;
    c.H = H;
    c.n_concepts = kb->n_concepts;
    c.n_roles = kb->n_roles;
    c.n_data = kb->n_props + kb->n_num;
    c.n_str = kb->n_str;
    c.n_patterns = kb->n_patterns;
    c.staged = use_staging(kb, kb->tuning);
    c.validated = false;
    c.z = dp::Sizes{kb->n, 4ull * kb->wp, kb->n_props, dnum, dstr, dcsr, kb->contain_words};
    const Tuning &tu = kb->tuning;
    c.warps = tu.warps;
    c.wpl = tu.wpl;
    c.rounds = tu.rounds;
    c.timeout_ms = tu.timeout_ms;
    c.wp = kb->wp;
    c.n_sms = (uint32_t)std::max(kb->n_sms, 0);
    c.flags = flags;

    // phase 1: validate, analyse and count per hypothesis; scan
    dp::count_kernel<<<grid_for(H, 128), 128, 0, st>>>(c, NI);
    dp::scan_kernel<<<1, dp::SCAN_THREADS, 0, st>>>(c);
    dp::Totals tot{};
    e = cudaGetLastError();
    if (!e) e = cudaMemcpyAsync(&tot, c.tot, sizeof tot, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return cuda_fail(e, "device planner (count, scan)");
    if (tot.err_hyp != 0xFFFFFFFFu)
        return fail(-(int)tot.err_code, "program " + std::to_string(tot.err_hyp) + " is not valid");
    if (tot.n_slots > REF_ID) return fail(HEDL_ERR_INVALID_ARG, "batch too large: more than 2^30 materialized intermediate sets");

    // phase 2: the image, laid out for at most NS groups and levels, zeroed, then filled
    const dp::Layout ub = dp::layout(tot.NS, tot.NS, tot.deps_n, tot.code_n, tot.NS, H, tot.n_slots, 4ull * kb->wp);
    void *img = nullptr;
    e = cudaMalloc(&img, ub.off_slots);
    if (e) return cuda_fail(e, "device plan image");
    std::unique_ptr<void, void (*)(void *)> img_guard(img, [](void *q) { cudaFree(q); });
    c.img = (uint8_t *)img;
    e = cudaMemsetAsync(img, 0, ub.off_slots, st);
    if (e) return cuda_fail(e, "device plan image");
    const uint64_t NS = tot.NS, n2 = dp::pow2_at_least(NS);
    dp::write_kernel<<<grid_for(H, 128), 128, 0, st>>>(c);
    dp::shape_kernel<<<1, dp::SCAN_THREADS, 0, st>>>(c);
    dp::key_kernel<<<grid_for(n2, 256), 256, 0, st>>>(c, n2);
    const uint64_t T = dp::BITONIC_TILE;
    const uint32_t tiles = (uint32_t)((n2 + T - 1) / T);
    dp::bitonic_tile_kernel<<<tiles, 1024, 0, st>>>(c.keys, n2, 2, std::min<uint64_t>(n2, T), T);
    for (uint64_t k = 2 * T; k <= n2; k <<= 1) {
        for (uint64_t j = k >> 1; j >= T; j >>= 1)
            dp::bitonic_global_kernel<<<grid_for(n2, 256), 256, 0, st>>>(c.keys, n2, j, k);
        dp::bitonic_tile_kernel<<<tiles, 1024, 0, st>>>(c.keys, n2, k, k, T >> 1);
    }
    dp::start_kernel<<<grid_for(NS, 256), 256, 0, st>>>(c);
    dp::group_scan_kernel<<<1, dp::SCAN_THREADS, 0, st>>>(c, gidx, Gd);
    dp::group_kernel<<<grid_for(NS, 256), 256, 0, st>>>(c, gidx, Gd, gbegin);
    dp::group_end_kernel<<<grid_for(NS, 256), 256, 0, st>>>(c, gidx, Gd, gbegin);
    dp::header_kernel<<<1, 1, 0, st>>>(c, Gd);
    const uint64_t span = std::max<uint64_t>(std::max<uint64_t>(NS, tot.code_n),
                                             std::max<uint64_t>(tot.deps_n, 4 + NS + 1 + 2ull * H));
    dp::assemble_kernel<<<grid_for(span, 256), 256, 0, st>>>(c, span);
    e = cudaGetLastError();
    PlanHeader hd{};
    std::vector<dp::HypCount> cnt(H);
    if (!e) e = cudaMemcpyAsync(&tot, c.tot, sizeof tot, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(&hd, img, sizeof hd, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(cnt.data(), c.cnt, sizeof(dp::HypCount) * H, cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) return cuda_fail(e, "device planner (write, sort, assemble)");
    if (tot.err_hyp == dp::ERR_BATCH)
        return fail(HEDL_ERR_INVALID_ARG, "batch too deep for the per-hypothesis planner: more than 16,384 dependency "
                                          "levels (nested role restrictions); plan it with hedl_plan_batch");
    if (tot.err_hyp != 0xFFFFFFFFu) return fail(HEDL_ERR_INVALID_ARG, "device planner: unexpected failure");
    if (tot.items >= 0xFFFFFFFFull) return fail(HEDL_ERR_INVALID_ARG, "batch too large: more than 2^32 work items");
    std::vector<uint32_t> level_items(tot.n_levels + 1);
    e = cudaMemcpy(level_items.data(), c.level_items, 4 * level_items.size(), cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(e, "device planner (level items)");

    auto *p = new PlanImpl();
    p->flags = flags;
    p->n_hyps = H;
    p->tuning = kb->tuning;
    p->staged = c.staged;
    p->info.n_hyps = H;
    p->info.total_insns = NI;
    p->info.n_nodes = NI;
    uint64_t model = 0;
    for (const dp::HypCount &n : cnt) {
        model += n.model;
        p->info.n_role_ops += n.n_role;
        p->info.n_data_ops += n.n_data;
        p->info.n_atom_loads += n.n_atom;
        p->max_stack = std::max(p->max_stack, n.max_depth);
    }
    if (p->max_stack > (uint32_t)STACK_MAX) {
        delete p;
        return fail(HEDL_ERR_BAD_PROGRAM, "internal: segment stack exceeds the device limit");
    }
    p->dev_image = img_guard.release();
    p->image_bytes = hd.off_slots;
    p->ctr_off = hd.off_ctr;
    p->ctr_bytes = (4 + (uint64_t)(tot.NS + 1) + 2ull * H) * 4;
    p->slots_off = hd.off_slots;
    p->ws_bytes = hd.off_ft;
    p->n_rgroups = 0;
    p->level_items = std::move(level_items);
    p->info.n_segments = hd.n_segs;
    p->info.n_slots = hd.n_slots;
    p->info.n_levels = hd.n_levels;
    p->info.n_items = hd.n_items;
    p->info.tile_words = hd.tile_words;
    p->info.warp_words = hd.warp_words;
    p->info.workspace_bytes = p->ws_bytes;
    p->info.image_bytes = p->image_bytes;
    p->info.model_bytes = model;
    *out = p;
    return HEDL_OK;
}

}  // namespace hedl

using namespace hedl;

extern "C" int hedl_plan_batch_device(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H,
                                      uint64_t n_insns, unsigned flags, hedl_stream s, hedl_plan **out) {
    if (!out) return fail(HEDL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!kb || !offs || !progs) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    PlanImpl *impl = nullptr;
    const int e = build_plan_device(kb, progs, offs, H, n_insns, flags, (cudaStream_t)s, &impl);
    if (e) return e;
    auto *p = new hedl_plan();
    p->impl = impl;
    *out = p;
    return HEDL_OK;
}

extern "C" int hedl_plan_batch_parallel(const hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H,
                                        unsigned flags, uint32_t n_threads, hedl_plan **out) {
    if (!out) return fail(HEDL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!kb || !offs || (H && offs[H] && !progs)) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    PlanImpl *impl = nullptr;
    const int e = build_plan_parallel(kb, progs, offs, H, flags, n_threads, &impl);
    if (e) return e;
    auto *p = new hedl_plan();
    p->impl = impl;
    *out = p;
    return HEDL_OK;
}
