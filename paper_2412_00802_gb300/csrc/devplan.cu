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
// The host driver runs steps 1-2 on several threads (the paper plans
// hypotheses in parallel on the CPU, Section V); the same functions are the
// body of a device-side planner (the paper's future work, Section VII).  The
// image equals the host planner's for the same flags, byte for byte.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
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
                const uint32_t ref = (op_of(progs[c]) == HEDL_OP_ATOM && !sc.mat[c]) ? a_of(progs[c])
                                                                                      : (REF_SLOT | read(c));
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

}  // namespace dp

namespace {

uint64_t put_bytes(std::vector<uint8_t> &img, const void *data, size_t n) {
    const uint64_t off = (img.size() + 255) & ~uint64_t(255);
    img.resize(off + n);
    if (n) memcpy(img.data() + off, data, n);
    return off;
}

template <typename T>
uint64_t put_vec(std::vector<uint8_t> &img, const std::vector<T> &v) {
    return put_bytes(img, v.data(), v.size() * sizeof(T));
}

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
    const bool staged = use_staging(kb, kb->tuning);
    if (!n_threads) n_threads = std::max(1u, std::thread::hardware_concurrency());
    {   // validation per hypothesis, in parallel; the first bad program is reported
        std::vector<int> err(H, 0);
        std::vector<std::string> why(H);
        parallel_for(H, n_threads, [&](uint32_t h) {
            err[h] = validate_program(kb, progs + offs[h], offs[h + 1] - offs[h], &why[h]);
        });
        for (uint32_t h = 0; h < H; ++h)
            if (err[h]) return fail(err[h], "program " + std::to_string(h) + ": " + why[h]);
    }
    const uint32_t NI = offs[H];
    std::vector<uint32_t> num_vals, str_vals, csr_edges;
    for (const DevNum &g : kb->num_host) num_vals.push_back(g.n_vals);
    for (const DevStr &g : kb->str_host) str_vals.push_back(g.n_vals);
    for (const DevCSR &g : kb->csr_host) csr_edges.push_back(g.n_edges);
    const dp::Sizes z{kb->n, 4ull * kb->wp, kb->n_props, num_vals.data(), str_vals.data(), csr_edges.data(),
                      kb->contain_words};
    std::vector<int32_t> k0(NI), k1(NI);
    std::vector<uint32_t> need(NI), slot(NI), level(NI), stk(NI);
    std::vector<uint8_t> mat(NI), state(NI);
    const dp::Scratch sc{k0.data(), k1.data(), need.data(), mat.data(), slot.data(), level.data(), stk.data(),
                         state.data()};

    // steps 1-2 (count): per hypothesis
    struct Count {
        uint32_t root = 0, n_mat = 0, mat_code = 0, mat_reads = 0, root_code = 0, root_reads = 0;
    };
    std::vector<Count> cnt(H);
    parallel_for(H, n_threads, [&](uint32_t h) {
        const uint32_t o0 = offs[h], o1 = offs[h + 1];
        Count &c = cnt[h];
        c.root = dp::analyze(progs, o0, o1, sc, staged);
        for (uint32_t k = o0; k < o1; ++k)
            if (mat[k]) {
                slot[k] = c.n_mat++;
                const dp::SegInfo s = dp::emit(progs, o0, sc, k, z, 0, nullptr, nullptr);
                level[k] = s.level;   // levels of earlier (operand) segments are set: node order
                c.mat_code += s.code_len;
                c.mat_reads += s.n_reads;
            }
        const dp::SegInfo r = dp::emit(progs, o0, sc, c.root, z, 0, nullptr, nullptr);
        c.root_code = r.code_len;
        c.root_reads = r.n_reads;
    });

    // step 3: prefix sums (materialised segments of every hypothesis first, then the roots)
    std::vector<uint32_t> slot_base(H), mcode(H), mdeps(H), rcode(H), rdeps(H);
    uint64_t n_slots = 0, code_n = 0, deps_n = 0;
    for (uint32_t h = 0; h < H; ++h) {
        slot_base[h] = (uint32_t)n_slots;
        mcode[h] = (uint32_t)code_n;
        mdeps[h] = (uint32_t)deps_n;
        n_slots += cnt[h].n_mat;
        code_n += cnt[h].mat_code;
        deps_n += cnt[h].mat_reads;
    }
    for (uint32_t h = 0; h < H; ++h) {
        rcode[h] = (uint32_t)code_n;
        rdeps[h] = (uint32_t)deps_n;
        code_n += cnt[h].root_code;
        deps_n += cnt[h].root_reads;
    }
    if (n_slots > REF_ID) return fail(HEDL_ERR_INVALID_ARG, "batch too large: more than 2^30 materialized intermediate sets");
    const uint32_t NS = (uint32_t)n_slots + H;
    std::vector<Seg> segs(NS);
    std::vector<DInsn> code(code_n);
    std::vector<uint32_t> deps(deps_n), seg_level(NS), seg_key(NS);
    std::vector<uint8_t> seg_walks(NS);
    struct Tally {
        uint64_t model = 0;
        uint32_t n_role = 0, n_data = 0, n_atom = 0, max_depth = 0;
    };
    std::vector<Tally> tally(H);

    // step 2 (write): per hypothesis, into its own ranges
    parallel_for(H, n_threads, [&](uint32_t h) {
        const uint32_t o0 = offs[h], o1 = offs[h + 1];
        uint32_t c_at = mcode[h], d_at = mdeps[h];
        Tally &t = tally[h];
        auto record = [&](uint32_t sidx, const dp::SegInfo &s, uint32_t c0, uint32_t d0, uint32_t out_slot,
                          uint32_t hyp) {
            Seg &g = segs[sidx];
            g.code_off = c0;
            g.code_len = s.code_len;
            g.out_slot = out_slot;
            g.hyp = hyp;
            g.dep_off = d0;
            g.dep_cnt = s.n_reads;
            g.filler = s.filler;
            g.kind = TASK_SEGMENT;
            seg_level[sidx] = s.level;
            seg_key[sidx] = s.key;
            seg_walks[sidx] = s.key != NO_FILLER;
            t.model += s.model;
            t.n_role += s.n_role;
            t.n_data += s.n_data;
            t.n_atom += s.n_atom;
            t.max_depth = std::max(t.max_depth, s.max_depth);
        };
        for (uint32_t k = o0; k < o1; ++k)
            if (mat[k]) {
                const dp::SegInfo s = dp::emit(progs, o0, sc, k, z, slot_base[h], code.data() + c_at, deps.data() + d_at);
                level[k] = s.level;
                record(slot_base[h] + slot[k], s, c_at, d_at, slot_base[h] + slot[k], NO_HYP);
                c_at += s.code_len;
                d_at += s.n_reads;
            }
        const dp::SegInfo r = dp::emit(progs, o0, sc, cnt[h].root, z, slot_base[h], code.data() + rcode[h],
                                       deps.data() + rdeps[h]);
        record((uint32_t)n_slots + h, r, rcode[h], rdeps[h], NO_SLOT, h);
        t.model += 2 * z.B + 16;
    });
    PlanImpl *p = new PlanImpl();
    p->flags = flags;
    p->n_hyps = H;
    p->tuning = kb->tuning;
    p->staged = staged;
    p->info.n_hyps = H;
    p->info.total_insns = NI;
    p->info.n_nodes = NI;
    uint64_t model = 0;
    for (const Tally &t : tally) {
        model += t.model;
        p->info.n_role_ops += t.n_role;
        p->info.n_data_ops += t.n_data;
        p->info.n_atom_loads += t.n_atom;
        p->max_stack = std::max(p->max_stack, t.max_depth);
    }
    if (p->max_stack > (uint32_t)STACK_MAX) {
        delete p;
        return fail(HEDL_ERR_BAD_PROGRAM, "internal: segment stack exceeds the device limit");
    }

    // step 4: tile shape (a reduction over levels), work queue (a stable sort)
    uint32_t n_levels = 0;
    for (uint32_t s = 0; s < NS; ++s) n_levels = std::max(n_levels, seg_level[s] + 1);
    const Tuning &t = p->tuning;
    uint32_t WW = 32, rounds = t.rounds;
    if (kb->n_sms > 0) {
        std::vector<uint32_t> segs_at(n_levels, 0);
        std::vector<uint8_t> walks_at(n_levels, 0);
        for (uint32_t s = 0; s < NS; ++s) {
            segs_at[seg_level[s]]++;
            walks_at[seg_level[s]] |= seg_walks[s];
        }
        uint64_t smin = UINT64_MAX;
        for (uint32_t L = 0; L < n_levels; ++L)
            if (walks_at[L]) smin = std::min<uint64_t>(smin, segs_at[L]);
        const uint64_t resident = 32ull * (uint64_t)kb->n_sms;
        if (smin != UINT64_MAX)
            while (WW > 4 && smin * kb->wp < 4ull * resident * WW * t.wpl) WW >>= 1;
        if (WW < 32) rounds = 1;
    }
    const uint32_t TW = t.warps * WW * t.wpl * rounds;
    const uint32_t n_tiles = (kb->wp + TW - 1) / TW;
    std::vector<uint32_t> order(NS);
    for (uint32_t s = 0; s < NS; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
        if (seg_level[x] != seg_level[y]) return seg_level[x] < seg_level[y];
        return seg_key[x] < seg_key[y];
    });
    std::vector<Group> groups;
    std::vector<uint32_t> gsegs;
    std::vector<uint32_t> level_items(n_levels + 1, 0);
    uint64_t items = 0;
    for (uint32_t k = 0; k < NS;) {
        const uint32_t s0 = order[k];
        Group g{};
        g.item_begin = (uint32_t)items;
        g.seg_begin = (uint32_t)gsegs.size();
        g.level = seg_level[s0];
        uint32_t k2 = k;
        while (k2 < NS && seg_level[order[k2]] == g.level && seg_key[order[k2]] == seg_key[s0]) gsegs.push_back(order[k2++]);
        g.n_segs = k2 - k;
        items += (uint64_t)g.n_segs * n_tiles;
        groups.push_back(g);
        level_items[g.level + 1] = (uint32_t)items;
        k = k2;
    }
    for (uint32_t l = 1; l <= n_levels; ++l) level_items[l] = std::max(level_items[l], level_items[l - 1]);
    if (items >= 0xFFFFFFFFull) {
        delete p;
        return fail(HEDL_ERR_INVALID_ARG, "batch too large: more than 2^32 work items");
    }

    // the image, laid out as the host planner lays it out
    std::vector<uint8_t> &img = p->image;
    img.resize(sizeof(PlanHeader));
    PlanHeader hd{};
    hd.n_items = (uint32_t)items;
    hd.n_segs = NS;
    hd.n_groups = (uint32_t)groups.size();
    hd.n_hyps = H;
    hd.n_tiles = n_tiles;
    hd.tile_words = TW;
    hd.warp_words = WW;
    hd.n_slots = (uint32_t)n_slots;
    hd.flags = flags;
    hd.n_levels = n_levels;
    hd.n_deps = (uint32_t)deps.size();
    hd.off_segs = put_vec(img, segs);
    hd.off_groups = put_vec(img, groups);
    hd.off_gsegs = put_vec(img, gsegs);
    hd.off_deps = put_vec(img, deps);
    hd.off_code = put_vec(img, code);
    hd.off_level_items = put_vec(img, level_items);
    hd.n_rgroups = 0;
    std::vector<uint32_t> zeros(4 + (NS + 1) + 2ull * H, 0);
    hd.off_ctr = put_vec(img, zeros);
    p->ctr_off = hd.off_ctr;
    p->ctr_bytes = zeros.size() * 4;
    hd.off_rgroups = put_bytes(img, nullptr, 0);
    img.resize((img.size() + 255) & ~size_t(255));
    hd.off_slots = img.size();
    hd.off_ft = (hd.off_slots + n_slots * 4ull * kb->wp + 255) & ~uint64_t(255);
    hd.timeout_ns = (uint64_t)t.timeout_ms * 1000000ull;
    memcpy(img.data(), &hd, sizeof hd);
    p->image_bytes = img.size();
    p->slots_off = hd.off_slots;
    p->ws_bytes = hd.off_ft;
    p->n_rgroups = 0;
    p->level_items = level_items;
    p->info.n_segments = NS;
    p->info.n_slots = (uint32_t)n_slots;
    p->info.n_levels = n_levels;
    p->info.n_items = (uint32_t)items;
    p->info.tile_words = TW;
    p->info.warp_words = WW;
    p->info.workspace_bytes = p->ws_bytes;
    p->info.image_bytes = p->image_bytes;
    p->info.model_bytes = model;
    *out = p;
    return HEDL_OK;
}

}  // namespace hedl

using namespace hedl;

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
