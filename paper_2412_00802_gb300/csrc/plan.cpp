// Host planner: turns a batch of postfix hypothesis programs into the device
// work queue executed by the segment interpreter (exec.cu).
//
// The paper builds an evaluation plan (a query plan fixing the order of the
// DL operations and their inputs) for each hypothesis on the CPU before it
// runs (Section IV), multi-threaded across a batch (Section V).  Here the plan
// of a whole batch is one DAG:
//   1. every program is decoded and validated, and its nodes are hash-consed
//      into one DAG shared by the batch (common sub-concepts are evaluated
//      once; AND/OR operands are put in canonical order and NOT NOT X folds to
//      X, which changes no instance set);
//   2. a node is materialized as a full bitset ("slot") if it is the filler
//      of a role restriction (a role restriction reads its filler at
//      arbitrary individuals, so the filler must exist over all individuals
//      first) or if it is used twice or more and its inline expansion holds a
//      role restriction (so that work is done once);
//   3. every materialized node and every hypothesis root becomes a segment:
//      a role-free boolean program whose leaves are atoms, data ranges,
//      slots and role restrictions over slots or concept rows;
//   4. role restrictions that share a role, direction and nesting depth with
//      another one become bit-sliced role groups (up to 32 per group, evaluated
//      by one transposed-filler walk) instead of living inside a segment;
//   5. tasks get levels (1 + the deepest producer of a slot they read) and
//      are grouped by (level, first role read); each group's work items are
//      (task, tile) pairs in tile-major order so that tasks sweeping the same
//      role stream the same CSR rows at about the same time;
//   6. the tile shape: 32 words per warp, or 16 / 8 / 4 with one round when a
//      level that walks a role holds too few tasks to fill the GPU.
#include <algorithm>
#include <cstring>
#include <unordered_map>

#include "hedl_internal.h"

namespace hedl {

namespace {

struct PNode {
    uint8_t op;
    uint8_t inv;
    uint16_t pad;
    uint32_t a;
    uint32_t b;
    int32_t k0, k1;
};

struct Key {
    uint64_t x, y;
    bool operator==(const Key &o) const { return x == o.x && y == o.y; }
};
struct KeyHash {
    size_t operator()(const Key &k) const {
        uint64_t h = k.x * 0x9E3779B97F4A7C15ull ^ (k.y + 0x632BE59BD9B4E019ull + (k.x << 6) + (k.x >> 2));
        h ^= h >> 31;
        h *= 0xBF58476D1CE4E5B9ull;
        return (size_t)(h ^ (h >> 29));
    }
};

inline bool is_role(uint32_t op) { return op >= HEDL_OP_EXISTS && op <= HEDL_OP_EXACTLY; }
inline bool is_data(uint32_t op) { return op >= HEDL_OP_DGE && op <= HEDL_OP_DEQ; }
inline bool is_str(uint32_t op) { return op == HEDL_OP_SEQ || op == HEDL_OP_SCONTAINS; }
// Algorithmic bytes of a data restriction on property id a: a one-value
// column (4N), or a numeric role's row pointers and values (4(N+1) + 4M).
inline uint64_t data_bytes(const hedl_kb *kb, uint32_t a, uint64_t N) {
    if (a < kb->n_props) return 4 * N;
    return 4 * (N + 1) + 4ull * kb->num_host[a - kb->n_props].n_vals;
}
// ... and of a string restriction: the role's row pointers and ids, plus
// SCONTAINS's row of the containment bitmap.
inline uint64_t str_bytes(const hedl_kb *kb, uint32_t op, uint32_t a, uint64_t N) {
    return 4 * (N + 1) + 4ull * kb->str_host[a].n_vals + (op == HEDL_OP_SCONTAINS ? 4 * kb->contain_words : 0);
}

inline int arity(uint32_t op) {
    if (op == HEDL_OP_ATOM || op == HEDL_OP_TOP || op == HEDL_OP_BOT || is_data(op) || is_str(op)) return 0;
    if (op == HEDL_OP_NOT || is_role(op)) return 1;
    if (op == HEDL_OP_AND || op == HEDL_OP_OR) return 2;
    return -1;
}

const char *op_name(uint32_t op) {
    static const char *names[] = {"?", "ATOM", "TOP", "BOT", "NOT", "AND", "OR", "EXISTS", "FORALL",
                                  "ATLEAST", "ATMOST", "EXACTLY", "DGE", "DLE", "DEQ", "SEQ", "SCONTAINS"};
    return op < 17 ? names[op] : "?";
}

}  // namespace

int validate_program(const hedl_kb *kb, const uint64_t *prog, uint32_t len, std::string *why) {
    if (len == 0) {
        *why = "empty program";
        return HEDL_ERR_BAD_PROGRAM;
    }
    int depth = 0;
    for (uint32_t k = 0; k < len; ++k) {
        uint64_t w = prog[k];
        uint32_t op = (uint32_t)(w & 0xFF);
        uint32_t a = (uint32_t)((w >> 16) & 0xFFFF);
        int ar = arity(op);
        char buf[160];
        if (ar < 0) {
            snprintf(buf, sizeof buf, "instruction %u: unknown op %u", k, op);
            *why = buf;
            return HEDL_ERR_BAD_PROGRAM;
        }
        if ((op == HEDL_OP_ATOM && a >= kb->n_concepts) || (is_role(op) && a >= kb->n_roles) ||
            (is_data(op) && a >= kb->n_props + kb->n_num) || (is_str(op) && a >= kb->n_str)) {
            snprintf(buf, sizeof buf, "instruction %u: %s names id %u, out of range", k, op_name(op), a);
            *why = buf;
            return HEDL_ERR_BAD_PROGRAM;
        }
        if (op == HEDL_OP_SCONTAINS && (uint32_t)(w >> 32) >= kb->n_patterns) {
            snprintf(buf, sizeof buf, "instruction %u: SCONTAINS names pattern %u, out of range", k,
                     (uint32_t)(w >> 32));
            *why = buf;
            return HEDL_ERR_BAD_PROGRAM;
        }
        if (depth < ar) {
            snprintf(buf, sizeof buf, "instruction %u: %s pops an empty stack", k, op_name(op));
            *why = buf;
            return HEDL_ERR_BAD_PROGRAM;
        }
        depth = depth - ar + 1;
        if (depth > HEDL_MAX_STACK) {
            snprintf(buf, sizeof buf, "instruction %u: more than %d operands on the stack", k, HEDL_MAX_STACK);
            *why = buf;
            return HEDL_ERR_BAD_PROGRAM;
        }
    }
    if (depth != 1) {
        *why = "program leaves " + std::to_string(depth) + " operands, not 1";
        return HEDL_ERR_BAD_PROGRAM;
    }
    return HEDL_OK;
}

uint64_t hash_programs(const uint64_t *progs, const uint32_t *offs, uint32_t H) {
    uint64_t h = 0xCBF29CE484222325ull ^ H;
    auto mix = [&](uint64_t v) {
        h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
        h *= 0x100000001B3ull;
    };
    for (uint32_t i = 0; i <= H; ++i) mix(offs[i]);
    for (uint32_t i = 0; i < offs[H]; ++i) mix(progs[i]);
    return h;
}

PlanImpl::~PlanImpl() = default;

namespace {

template <class T>
uint64_t put(std::vector<uint8_t> &img, const std::vector<T> &v) {
    uint64_t off = (img.size() + 255) & ~uint64_t(255);
    img.resize(off + v.size() * sizeof(T));
    if (!v.empty()) memcpy(img.data() + off, v.data(), v.size() * sizeof(T));
    return off;
}

}  // namespace

int build_plan(const hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, unsigned flags,
               PlanImpl **out) {
    *out = nullptr;
    if (H == 0) return fail(HEDL_ERR_INVALID_ARG, "empty batch (H = 0)");
    if (offs[0] != 0) return fail(HEDL_ERR_INVALID_ARG, "offs[0] must be 0");
    for (uint32_t h = 0; h < H; ++h) {
        if (offs[h + 1] < offs[h]) return fail(HEDL_ERR_INVALID_ARG, "offs must be non-decreasing");
        std::string why;
        int e = validate_program(kb, progs + offs[h], offs[h + 1] - offs[h], &why);
        if (e) return fail(e, "program " + std::to_string(h) + ": " + why);
    }
    auto *p = new PlanImpl();
    p->flags = flags;
    p->n_hyps = H;
    p->tuning = kb->tuning;
    const uint64_t N = kb->n, B = 4ull * kb->wp;
    p->info.n_hyps = H;
    p->info.total_insns = offs[H];

    if (flags & HEDL_PLAIN) {
        // One launch per operation: keep the programs; the stack of the
        // deepest program sizes the workspace.
        p->progs.assign(progs, progs + offs[H]);
        p->offs.assign(offs, offs + H + 1);
        uint32_t maxd = 1;
        uint64_t mb = 0;
        for (uint32_t h = 0; h < H; ++h) {
            int d = 0;
            for (uint32_t k = offs[h]; k < offs[h + 1]; ++k) {
                uint32_t op = (uint32_t)(progs[k] & 0xFF);
                uint32_t a = (uint32_t)((progs[k] >> 16) & 0xFFFF);
                d = d - arity(op) + 1;
                maxd = std::max<uint32_t>(maxd, (uint32_t)d);
                if (op == HEDL_OP_ATOM) mb += B, p->info.n_atom_loads++;
                else if (is_data(op)) mb += data_bytes(kb, a, N), p->info.n_data_ops++;
                else if (is_str(op)) mb += str_bytes(kb, op, a, N), p->info.n_data_ops++;
                else if (is_role(op)) mb += 4 * (N + 1) + 4ull * kb->role_edges[a] + 2 * B, p->info.n_role_ops++;
            }
            mb += 2 * B + 16;  // scoring
        }
        p->plain_depth = maxd;
        p->info.model_bytes = mb;
        // workspace: header page, accumulators [H][2], stack rows
        uint64_t acc_off = 256;
        uint64_t rows_off = (acc_off + 8ull * H + 255) & ~uint64_t(255);
        p->ws_bytes = rows_off + (uint64_t)(maxd + 1) * B;
        p->info.workspace_bytes = p->ws_bytes;
        p->info.n_levels = 0;
        *out = p;
        return HEDL_OK;
    }

    const bool cse = !(flags & HEDL_NO_CSE);
    std::vector<PNode> nodes;
    nodes.reserve(offs[H] + 16);
    std::unordered_map<Key, int32_t, KeyHash> memo;
    memo.reserve(cse ? offs[H] * 2 + 16 : 0);
    auto make = [&](PNode n) -> int32_t {
        // canonical form: ignored fields zeroed, commutative operands ordered
        if (!is_role(n.op)) n.inv = 0;
        if (!(n.op == HEDL_OP_ATOM || is_role(n.op) || is_data(n.op) || is_str(n.op))) n.a = 0;
        if (!(n.op == HEDL_OP_ATLEAST || n.op == HEDL_OP_ATMOST || n.op == HEDL_OP_EXACTLY || is_data(n.op) ||
              is_str(n.op)))
            n.b = 0;
        if (cse) {
            if ((n.op == HEDL_OP_AND || n.op == HEDL_OP_OR) && n.k0 > n.k1) std::swap(n.k0, n.k1);
            if (n.op == HEDL_OP_NOT && nodes[n.k0].op == HEDL_OP_NOT) return nodes[n.k0].k0;
            Key k{(uint64_t)n.op | ((uint64_t)n.inv << 8) | ((uint64_t)n.a << 16) | ((uint64_t)n.b << 32),
                  (uint64_t)(uint32_t)n.k0 | ((uint64_t)(uint32_t)n.k1 << 32)};
            auto it = memo.find(k);
            if (it != memo.end()) return it->second;
            memo.emplace(k, (int32_t)nodes.size());
        }
        nodes.push_back(n);
        return (int32_t)nodes.size() - 1;
    };

    std::vector<int32_t> roots(H);
    std::vector<int32_t> st;
    for (uint32_t h = 0; h < H; ++h) {
        st.clear();
        for (uint32_t k = offs[h]; k < offs[h + 1]; ++k) {
            uint64_t w = progs[k];
            PNode n{};
            n.op = (uint8_t)(w & 0xFF);
            n.inv = (uint8_t)((w >> 8) & 1);
            n.a = (uint32_t)((w >> 16) & 0xFFFF);
            n.b = (uint32_t)(w >> 32);
            n.k0 = n.k1 = -1;
            int ar = arity(n.op);
            if (ar == 2) {
                n.k1 = st.back();
                st.pop_back();
                n.k0 = st.back();
                st.pop_back();
            } else if (ar == 1) {
                n.k0 = st.back();
                st.pop_back();
            }
            st.push_back(make(n));
        }
        roots[h] = st.back();
    }
    const uint32_t NN = (uint32_t)nodes.size();
    p->info.n_nodes = NN;

    // reference counts (parents + hypothesis roots)
    std::vector<uint32_t> refc(NN, 0);
    for (uint32_t i = 0; i < NN; ++i) {
        if (nodes[i].k0 >= 0) refc[nodes[i].k0]++;
        if (nodes[i].k1 >= 0) refc[nodes[i].k1]++;
    }
    for (uint32_t h = 0; h < H; ++h) refc[roots[h]]++;

    // materialization (children are created before parents, so index order
    // is a topological order)
    std::vector<uint8_t> mat(NN, 0);
    for (uint32_t i = 0; i < NN; ++i)
        if (is_role(nodes[i].op) && nodes[nodes[i].k0].op != HEDL_OP_ATOM) mat[nodes[i].k0] = 1;
    // Bit-sliced role restrictions: each is materialized and evaluated by its
    // role group's shared walk (counting ones need n <= SLICE_MAX_N).  A walk
    // shared by one restriction only costs a transpose and a 32-times larger
    // filler, so by default a restriction is sliced only when another one has
    // the same role, direction and depth (role restrictions nested below it,
    // itself included), the depth standing in for the level it becomes ready at.
    const bool sliced = !(flags & HEDL_NO_SLICE);
    std::vector<uint8_t> sl(NN, 0);
    std::vector<uint32_t> rdepth(NN, 0);
    if (sliced) {
        auto eligible = [&](const PNode &n) {
            return is_role(n.op) && (n.op == HEDL_OP_EXISTS || n.op == HEDL_OP_FORALL || n.b <= SLICE_MAX_N);
        };
        std::unordered_map<uint64_t, uint32_t> same;
        for (uint32_t i = 0; i < NN; ++i) {
            const PNode &n = nodes[i];
            uint32_t d = 0;
            if (n.k0 >= 0) d = std::max(d, rdepth[n.k0]);
            if (n.k1 >= 0) d = std::max(d, rdepth[n.k1]);
            rdepth[i] = d + (is_role(n.op) ? 1u : 0u);
            if (eligible(n)) same[((uint64_t)rdepth[i] << 32) | (n.a * 2u + n.inv)]++;
        }
        for (uint32_t i = 0; i < NN; ++i) {
            const PNode &n = nodes[i];
            if (eligible(n) &&
                ((flags & HEDL_SLICE_ALL) || same[((uint64_t)rdepth[i] << 32) | (n.a * 2u + n.inv)] >= 2)) {
                sl[i] = 1;
                mat[i] = 1;
            }
        }
    }
    std::vector<uint8_t> role_inline(NN, 0);
    std::vector<uint32_t> need(NN, 1);
    for (uint32_t i = 0; i < NN; ++i) {
        const PNode &n = nodes[i];
        auto ri = [&](int32_t c) { return c >= 0 && !mat[c] && role_inline[c]; };
        role_inline[i] = is_role(n.op) || ri(n.k0) || ri(n.k1);
        if (!mat[i] && refc[i] >= 2 && role_inline[i] && n.op != HEDL_OP_ATOM) mat[i] = 1;
        // stack need (Sethi-Ullman), materialized children count as leaves
        auto nd = [&](int32_t c) -> uint32_t { return mat[c] ? 1u : need[c]; };
        if (n.op == HEDL_OP_NOT) need[i] = nd(n.k0);
        else if (n.op == HEDL_OP_AND || n.op == HEDL_OP_OR) {
            uint32_t a = nd(n.k0), b = nd(n.k1);
            uint32_t v = a == b ? a + 1 : std::max(a, b);
            if (v > (uint32_t)STACK_MAX - 1) {   // keep every segment within the device stack
                mat[a >= b ? n.k0 : n.k1] = 1;
                a = nd(n.k0);
                b = nd(n.k1);
                v = a == b ? a + 1 : std::max(a, b);
            }
            need[i] = v;
        } else need[i] = 1;
    }

    // With staged fillers each segment may read one role restriction (its
    // filler is copied to shared memory once per work item): any further role
    // restriction in a segment's inline expansion becomes its own segment.
    const bool staged = use_staging(kb, kb->tuning);
    p->staged = staged;
    if (staged) {
        std::vector<int32_t> seg_roots;
        for (uint32_t i = 0; i < NN; ++i)
            if (mat[i]) seg_roots.push_back((int32_t)i);
        for (uint32_t h = 0; h < H; ++h)
            if (!mat[roots[h]]) seg_roots.push_back(roots[h]);
        std::vector<int32_t> dfs;
        for (int32_t r : seg_roots) {
            bool kept = false;
            dfs.clear();
            dfs.push_back(r);
            while (!dfs.empty()) {
                int32_t i = dfs.back();
                dfs.pop_back();
                if (i != r && mat[i]) continue;
                const PNode &n = nodes[i];
                if (is_role(n.op)) {
                    if (kept && i != r) mat[i] = 1;
                    kept = true;
                    continue;   // its filler is a slot or a concept row, not inline
                }
                if (n.k1 >= 0) dfs.push_back(n.k1);
                if (n.k0 >= 0) dfs.push_back(n.k0);
            }
        }
    }

    // slots and segments
    std::vector<uint32_t> slot_of(NN, NO_SLOT);
    uint32_t n_slots = 0;
    for (uint32_t i = 0; i < NN; ++i)
        if (mat[i]) slot_of[i] = n_slots++;
    if (n_slots > REF_ID) {
        delete p;
        return fail(HEDL_ERR_INVALID_ARG, "batch too large: more than 2^30 materialized intermediate sets");
    }
    std::vector<Seg> segs;
    std::vector<DInsn> code;
    std::vector<std::vector<uint32_t>> seg_slots_read;
    std::vector<uint32_t> seg_of_slot(n_slots, 0);
    std::vector<uint32_t> role_key;  // first role read, for grouping
    // Algorithmic bytes, the per-operation model (no credit for sharing a CSR
    // walk or for caches): an atom read B (a role restriction's filler concept
    // included), a data range 4N, a role restriction 4(N+1) + 4E + 2B (row
    // pointers, columns, filler written and read), a hypothesis score
    // 2B + 16, over the operations left after common sub-concepts are shared.
    uint64_t model = 0;

    std::vector<int32_t> work;
    auto emit_segment = [&](int32_t root, uint32_t out_slot, uint32_t hyp) {
        Seg s{};
        s.code_off = (uint32_t)code.size();
        s.out_slot = out_slot;
        s.hyp = hyp;
        s.filler = NO_FILLER;
        std::vector<uint32_t> reads;
        uint32_t rk = 0xFFFFFFFFu;
        // iterative post-order emission, larger stack need first
        struct Frame { int32_t n; int state; };
        std::vector<Frame> fr;
        fr.push_back({root, 0});
        int depth = 0, maxdepth = 0;
        while (!fr.empty()) {
            Frame &f = fr.back();
            int32_t i = f.n;
            const PNode &n = nodes[i];
            bool leafish = (i != root && mat[i]) || arity(n.op) == 0 || is_role(n.op);
            if (leafish) {
                DInsn d{};
                if (i != root && mat[i]) {
                    d.op = D_SLOT;
                    d.ref = slot_of[i];
                    reads.push_back(slot_of[i]);   // bytes counted with the restriction that made it
                } else if (n.op == HEDL_OP_ATOM) {
                    d.op = D_ATOM;
                    d.a = n.a;
                    model += B;
                    p->info.n_atom_loads++;
                } else if (n.op == HEDL_OP_TOP || n.op == HEDL_OP_BOT) {
                    d.op = n.op;
                } else if (is_data(n.op)) {
                    const bool num = n.a >= kb->n_props;   // a numeric concrete role
                    d.op = D_DATA | (n.op << 16) | (num ? 1u << 8 : 0u);
                    d.a = num ? n.a - kb->n_props : n.a;
                    d.b = n.b;
                    model += data_bytes(kb, n.a, N);
                    p->info.n_data_ops++;
                } else if (is_str(n.op)) {   // a string concrete role
                    d.op = D_DATA | (n.op << 16) | (1u << 9);
                    d.a = n.a;
                    d.b = n.b;
                    model += str_bytes(kb, n.op, n.a, N);
                    p->info.n_data_ops++;
                } else {  // role restriction
                    int32_t c = n.k0;
                    d.op = D_ROLE | ((uint32_t)n.inv << 8) | ((uint32_t)n.op << 16);
                    d.a = n.a;
                    d.b = n.b;
                    if (nodes[c].op == HEDL_OP_ATOM && !mat[c]) {
                        d.ref = nodes[c].a;
                        model += B;   // the filler concept's row: an atom leaf of the plain method
                    } else {
                        d.ref = REF_SLOT | slot_of[c];
                        reads.push_back(slot_of[c]);
                    }
                    if (rk == 0xFFFFFFFFu) rk = n.a * 2 + n.inv;
                    if (s.filler == NO_FILLER) s.filler = d.ref | (n.op == HEDL_OP_FORALL ? REF_NEG : 0u);
                    const DevCSR &g = kb->csr_host[2 * n.a + n.inv];
                    model += 4 * (N + 1) + 4ull * g.n_edges + 2 * B;
                    p->info.n_role_ops++;
                }
                code.push_back(d);
                depth++;
                maxdepth = std::max(maxdepth, depth);
                fr.pop_back();
                continue;
            }
            if (n.op == HEDL_OP_NOT) {
                if (f.state == 0) {
                    f.state = 1;
                    fr.push_back({n.k0, 0});
                } else {
                    DInsn d{};
                    d.op = D_NOT;
                    code.push_back(d);
                    fr.pop_back();
                }
                continue;
            }
            // AND / OR
            auto nd = [&](int32_t c) -> uint32_t { return mat[c] ? 1u : need[c]; };
            int32_t first = nd(n.k0) >= nd(n.k1) ? n.k0 : n.k1;
            int32_t second = first == n.k0 ? n.k1 : n.k0;
            if (f.state == 0) {
                f.state = 1;
                fr.push_back({first, 0});
            } else if (f.state == 1) {
                f.state = 2;
                fr.push_back({second, 0});
            } else {
                DInsn d{};
                d.op = n.op;
                code.push_back(d);
                depth--;
                fr.pop_back();
            }
        }
        s.code_len = (uint32_t)code.size() - s.code_off;
        p->max_stack = std::max(p->max_stack, (uint32_t)maxdepth);
        if (hyp != NO_HYP) model += 2 * B + 16;
        std::sort(reads.begin(), reads.end());
        reads.erase(std::unique(reads.begin(), reads.end()), reads.end());
        seg_slots_read.push_back(reads);
        role_key.push_back(rk);
        segs.push_back(s);
    };
    for (uint32_t i = 0; i < NN; ++i)
        if (mat[i] && !sl[i]) {
            seg_of_slot[slot_of[i]] = (uint32_t)segs.size();
            emit_segment((int32_t)i, slot_of[i], NO_HYP);
        }
    for (uint32_t h = 0; h < H; ++h) {
        if (mat[roots[h]]) {  // the root is already a slot: the segment reads it
            Seg s{};
            s.code_off = (uint32_t)code.size();
            s.code_len = 1;
            s.out_slot = NO_SLOT;
            s.hyp = h;
            s.filler = NO_FILLER;
            DInsn d{};
            d.op = D_SLOT;
            d.ref = slot_of[roots[h]];
            code.push_back(d);
            model += 2 * B + 16;
            seg_slots_read.push_back({slot_of[roots[h]]});
            role_key.push_back(0xFFFFFFFFu);
            segs.push_back(s);
            p->max_stack = std::max(p->max_stack, 1u);
        } else {
            emit_segment(roots[h], NO_SLOT, h);
        }
    }
    if (p->max_stack > (uint32_t)STACK_MAX) {
        delete p;
        return fail(HEDL_ERR_BAD_PROGRAM, "internal: segment stack exceeds the device limit");
    }
    const uint32_t NSEG = (uint32_t)segs.size();
    const uint64_t FT_PART = 4ull * 32ull * kb->wp;   // one FT word per individual (>= 4 N bytes)

    // Sliced restrictions are grouped by (role depth, role, direction): one
    // group key per distinct triple, in a dense numbering.
    std::vector<uint32_t> key_of(NN, 0xFFFFFFFFu);
    std::vector<uint64_t> key_val;
    uint32_t max_rd = 0;
    {
        std::unordered_map<uint64_t, uint32_t> ids;
        for (uint32_t i = 0; i < NN; ++i) {
            if (!sl[i]) continue;
            const uint64_t k = ((uint64_t)rdepth[i] << 32) | (nodes[i].a * 2u + nodes[i].inv);
            auto it = ids.find(k);
            if (it == ids.end()) {
                it = ids.emplace(k, (uint32_t)key_val.size()).first;
                key_val.push_back(k);
            }
            key_of[i] = it->second;
            max_rd = std::max(max_rd, rdepth[i]);
        }
    }

    // Production level of every slot and level of every segment, in node order
    // (children first).  A segment reading nothing is at level 0 and one level
    // above the slots it reads.  A sliced role restriction is ready one level
    // above its filler's transpose, which runs one level above the filler's
    // producer (level 0 for a concept row); all restrictions of a group key
    // walk together, at the level of the group's last-ready one.  A filler
    // holds only restrictions of smaller role depth, so the levels of depth d
    // are final once those of depths below d are: one pass per depth fixes
    // them in turn, and a last pass sets every level.
    std::vector<uint32_t> slot_level(n_slots, 0), seg_level(NSEG, 0);
    std::vector<uint32_t> group_level(key_val.size(), 0);
    auto seg_lvl = [&](uint32_t sidx) {
        uint32_t lvl = 0;
        for (uint32_t sl2 : seg_slots_read[sidx]) lvl = std::max(lvl, slot_level[sl2] + 1);
        return lvl;
    };
    for (uint32_t d = 1; d <= max_rd + 1; ++d) {
        std::vector<uint32_t> ready(key_val.size(), 0);
        for (uint32_t i = 0; i < NN; ++i) {
            if (!mat[i]) continue;
            if (sl[i]) {
                const int32_t f = nodes[i].k0;
                const bool concept_filler = nodes[f].op == HEDL_OP_ATOM && !mat[f];
                const uint32_t own = concept_filler ? 1u : slot_level[slot_of[f]] + 2u;
                uint32_t lvl = own;
                if (rdepth[i] < d) lvl = group_level[key_of[i]];
                else if (rdepth[i] == d) ready[key_of[i]] = std::max(ready[key_of[i]], own);
                slot_level[slot_of[i]] = lvl;
            } else {
                const uint32_t sidx = seg_of_slot[slot_of[i]];
                seg_level[sidx] = seg_lvl(sidx);
                slot_level[slot_of[i]] = seg_level[sidx];
            }
        }
        for (size_t k = 0; k < key_val.size(); ++k)
            if ((key_val[k] >> 32) == d) group_level[k] = ready[k];
        if (!sliced) break;
    }
    for (uint32_t sidx = 0; sidx < NSEG; ++sidx)
        if (segs[sidx].hyp != NO_HYP) seg_level[sidx] = seg_lvl(sidx);

    // role groups: sliced restrictions keyed by (role depth, role, direction), up to
    // SLICES * MAX_PARTS at a time (one FT word per 32 of them)
    std::vector<RGroup> rgroups;
    std::vector<uint32_t> task_level(seg_level);
    std::vector<uint32_t> task_key(role_key);
    std::vector<std::vector<uint32_t>> task_reads(seg_slots_read);
    uint64_t ft_bytes = 0;
    {
        std::vector<std::pair<uint64_t, uint32_t>> keyed;   // ((level << 32) | role2, node)
        for (uint32_t i = 0; i < NN; ++i)
            if (sl[i]) keyed.push_back({((uint64_t)slot_level[slot_of[i]] << 32) | (nodes[i].a * 2 + nodes[i].inv), i});
        std::stable_sort(keyed.begin(), keyed.end(),
                         [](const std::pair<uint64_t, uint32_t> &x, const std::pair<uint64_t, uint32_t> &y) {
                             return x.first < y.first;
                         });
        for (size_t k = 0; k < keyed.size();) {
            size_t k2 = k;
            while (k2 < keyed.size() && keyed[k2].first == keyed[k].first && k2 - k < SLICES * MAX_PARTS) ++k2;
            RGroup g{};
            g.role2 = (uint32_t)(keyed[k].first & 0xFFFFFFFFu);
            g.n = (uint32_t)(k2 - k);
            g.parts = g.n > SLICES ? MAX_PARTS : 1u;
            std::vector<uint32_t> reads;
            for (size_t q = k; q < k2; ++q) {
                const uint32_t i = keyed[q].second;
                const PNode &n = nodes[i];
                const int32_t f = n.k0;
                const uint32_t s_ = (uint32_t)(q - k);
                if (nodes[f].op == HEDL_OP_ATOM && !mat[f]) {
                    g.filler[s_] = nodes[f].a;
                    model += B;   // the filler concept's row
                } else {
                    g.filler[s_] = REF_SLOT | slot_of[f];
                    reads.push_back(slot_of[f]);
                }
                if (n.op == HEDL_OP_FORALL) g.filler[s_] |= REF_NEG;
                g.out[s_] = slot_of[i];
                for (uint32_t v = 0; v < 8; ++v) {
                    bool holds;
                    switch (n.op) {
                    case HEDL_OP_EXISTS: holds = v >= 1; break;
                    case HEDL_OP_FORALL: holds = v == 0; break;   // successors outside C
                    case HEDL_OP_ATLEAST: holds = v >= n.b; break;
                    case HEDL_OP_ATMOST: holds = v <= n.b; break;
                    default: holds = v == n.b; break;
                    }
                    if (holds) g.want[s_ / SLICES][v] |= 1u << (s_ % SLICES);
                }
                p->info.n_role_ops++;
            }
            std::sort(reads.begin(), reads.end());
            reads.erase(std::unique(reads.begin(), reads.end()), reads.end());
            const uint32_t gi = (uint32_t)rgroups.size();
            const uint32_t wl = (uint32_t)(keyed[k].first >> 32);
            // transpose task, then walk task
            Seg t{};
            t.code_off = gi;
            t.out_slot = NO_SLOT;
            t.hyp = NO_HYP;
            t.filler = NO_FILLER;
            t.kind = TASK_TRANSPOSE;
            segs.push_back(t);
            task_level.push_back(wl - 1);
            task_key.push_back(g.role2 | 0x80000000u);
            task_reads.push_back(reads);
            Seg w = t;
            w.kind = TASK_WALK;
            const uint32_t walk_task = (uint32_t)segs.size();
            segs.push_back(w);
            task_level.push_back(wl);
            task_key.push_back(g.role2);
            task_reads.push_back({});
            for (uint32_t s_ = 0; s_ < g.n; ++s_) seg_of_slot[g.out[s_]] = walk_task;
            const DevCSR &csr = kb->csr_host[g.role2];
            model += (uint64_t)g.n * (4 * (N + 1) + 4ull * csr.n_edges + 2 * B);
            g.ft_off = ft_bytes;   // relative to the FT region until the slots are placed
            ft_bytes += g.parts * FT_PART;
            rgroups.push_back(g);
            k = k2;
        }
    }
    const uint32_t NS = (uint32_t)segs.size();

    // dependencies (the producer task of every slot read; a walk waits for its transpose)
    std::vector<uint32_t> deps;
    uint32_t n_levels = 0;
    for (uint32_t s_ = 0; s_ < NS; ++s_) {
        segs[s_].dep_off = (uint32_t)deps.size();
        if (segs[s_].kind == TASK_WALK) {
            deps.push_back(s_ - 1);
        } else {
            for (uint32_t sl2 : task_reads[s_]) deps.push_back(seg_of_slot[sl2]);
        }
        segs[s_].dep_cnt = (uint32_t)deps.size() - segs[s_].dep_off;
        n_levels = std::max(n_levels, task_level[s_] + 1);
    }
    if (flags & HEDL_TEST_UNSAT_DEP) {
        // the last segment additionally waits on a counter past the real
        // ones, which nothing ever increments
        segs[NSEG - 1].dep_off = (uint32_t)deps.size();
        segs[NSEG - 1].dep_cnt = 1;
        deps.push_back(NS);
    }

    // Tile shape.  A warp covers 32 words a round by default.  When some level
    // that walks a role holds only a few segments (a small batch, a single
    // hypothesis), its tiles would keep only a fraction of the resident warps
    // busy, each walking 32 words in sequence: then a warp covers fewer words
    // (down to 4, one round per item) so that the level spreads over about
    // four times as many warp-rounds as there are resident warps (32 per SM at
    // 64 registers), which also balances rows of very different degree.  Role
    // groups walk 32 words per warp and keep the default shape.
    const Tuning &t = p->tuning;
    uint32_t WW = 32, rounds = t.rounds;
    if (rgroups.empty() && kb->n_sms > 0) {
        std::vector<uint32_t> segs_at(n_levels, 0);
        std::vector<uint8_t> walks_at(n_levels, 0);
        for (uint32_t s_ = 0; s_ < NS; ++s_) {
            const uint32_t L = task_level[s_];
            segs_at[L]++;
            for (uint32_t pc = 0; pc < segs[s_].code_len; ++pc)
                if ((code[segs[s_].code_off + pc].op & 0xFFu) == D_ROLE) walks_at[L] = 1;
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
        if (task_level[x] != task_level[y]) return task_level[x] < task_level[y];
        return task_key[x] < task_key[y];
    });
    std::vector<Group> groups;
    std::vector<uint32_t> gsegs;
    std::vector<uint32_t> level_items(n_levels + 1, 0);
    uint64_t items = 0;
    for (uint32_t k = 0; k < NS;) {
        uint32_t s0 = order[k];
        Group g{};
        g.item_begin = (uint32_t)items;
        g.seg_begin = (uint32_t)gsegs.size();
        g.level = task_level[s0];
        uint32_t k2 = k;
        while (k2 < NS && task_level[order[k2]] == g.level && task_key[order[k2]] == task_key[s0]) {
            gsegs.push_back(order[k2]);
            ++k2;
        }
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

    // image: header, tables, counters; then the slots
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
    hd.n_slots = n_slots;
    hd.flags = flags;
    hd.n_levels = n_levels;
    hd.n_deps = (uint32_t)deps.size();
    hd.off_segs = put(img, segs);
    hd.off_groups = put(img, groups);
    hd.off_gsegs = put(img, gsegs);
    hd.off_deps = put(img, deps);
    hd.off_code = put(img, code);
    hd.off_level_items = put(img, level_items);
    hd.n_rgroups = (uint32_t)rgroups.size();
    // counters: Counters + done[NS + 1] + acc[H][2]
    std::vector<uint32_t> zeros(4 + (NS + 1) + 2ull * H, 0);
    hd.off_ctr = put(img, zeros);
    p->ctr_off = hd.off_ctr;
    p->ctr_bytes = zeros.size() * 4;
    hd.off_rgroups = put(img, rgroups);   // FT offsets patched below, once the slots are placed
    img.resize((img.size() + 255) & ~size_t(255));
    hd.off_slots = img.size();
    hd.off_ft = (hd.off_slots + (uint64_t)n_slots * B + 255) & ~uint64_t(255);
    for (size_t g = 0; g < rgroups.size(); ++g) rgroups[g].ft_off += hd.off_ft;
    if (!rgroups.empty()) memcpy(img.data() + hd.off_rgroups, rgroups.data(), rgroups.size() * sizeof(RGroup));
    hd.timeout_ns = (uint64_t)t.timeout_ms * 1000000ull;
    memcpy(img.data(), &hd, sizeof hd);
    p->image_bytes = img.size();
    p->slots_off = hd.off_slots;
    p->ws_bytes = hd.off_ft + ft_bytes;
    p->n_rgroups = (uint32_t)rgroups.size();
    p->info.n_role_groups = (uint32_t)rgroups.size();
    p->level_items = level_items;

    p->info.n_segments = NS;
    p->info.n_slots = n_slots;
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
