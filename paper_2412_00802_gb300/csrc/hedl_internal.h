// Library-private declarations shared by the host planner (plan.cpp), the
// C-ABI layer (api.cu) and the device kernels (exec.cu, plain.cu, kb.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hedl.h"

namespace hedl {

// ------------------------------------------------------------------ device-side KB view
struct DevCSR {
    const uint32_t *rp;    // [n+1]
    const uint32_t *col;   // [E]
    uint32_t n_edges;
    uint32_t pad;
};

// A numeric concrete role: CSR of values over subjects.
struct DevNum {
    const uint32_t *rp;    // [n+1]
    const float *vals;     // [n_vals]
    uint32_t n_vals;
    uint32_t pad;
};

// A string concrete role: CSR of interned string ids over subjects.
struct DevStr {
    const uint32_t *rp;    // [n+1]
    const uint32_t *ids;   // [n_vals], each < n_strings
    uint32_t n_vals;
    uint32_t pad;
};

// Passed by value to every kernel.
struct KBView {
    const uint32_t *concepts;    // [C][wp]
    const DevCSR *csr;           // device [2*R]: role r forward at 2r, inverse at 2r+1
    const DevNum *num;           // device [Q]: the numeric concrete roles
    const DevStr *str;           // device [S]: the string concrete roles
    const uint32_t *contain;     // [n_patterns][contain_words]: bit i of row k = string i contains pattern k
    uint64_t contain_words;
    const float *props;          // [P][prop_stride]
    uint64_t prop_stride;
    const uint32_t *pos;         // [wp] or null
    const uint32_t *neg;
    uint32_t *status;            // device status word owned by the handle
    uint32_t n, w, wp;           // individuals, valid words, row words
    uint32_t n_pos, n_neg;
};

// status word bits (device)
enum : uint32_t { ST_TIMEOUT = 1u, ST_DEVICE_CHECK = 2u };

// ------------------------------------------------------------------ segment code
// One 16-byte instruction of a segment program (a role-free boolean
// expression whose leaves may be role restrictions over materialized fillers).
enum : uint32_t {
    D_ATOM = 1, D_TOP = 2, D_BOT = 3, D_NOT = 4, D_AND = 5, D_OR = 6,
    D_ROLE = 7,      // aux = kind (HEDL_OP_EXISTS..EXACTLY), a = role, flags bit0 = inverse, b = n
    D_DATA = 12,     // aux = the op (HEDL_OP_DGE/DLE/DEQ/SEQ/SCONTAINS); bits 8/9 of the op
                     // word clear: a = one-value property, b = float bits; bit 8: a = numeric
                     // role, b = float bits; bit 9: a = string role, b = string / pattern id
    D_SLOT = 32      // a materialized bitset: ref = slot index
};
constexpr uint32_t REF_SLOT = 0x80000000u;   // filler ref: slot (low bits) vs concept id
constexpr uint32_t REF_NEG = 0x40000000u;    // Seg.filler only: stage the complement (FORALL)
constexpr uint32_t REF_ID = 0x3FFFFFFFu;     // slot or concept id bits of a ref

struct DInsn {
    uint32_t op;     // D_*
    uint32_t a;      // concept / role / property id
    uint32_t b;      // n or threshold bits
    uint32_t ref;    // D_ROLE: filler ref; D_SLOT: slot; bits 16..23 of op word: aux, bit 8: inverse
};
inline uint32_t dop(uint32_t w) { return w & 0xFF; }

constexpr uint32_t NO_SLOT = 0xFFFFFFFFu;
constexpr uint32_t NO_HYP = 0xFFFFFFFFu;

constexpr uint32_t NO_FILLER = 0xFFFFFFFFu;

// A task of the work queue: a segment (kind 0), or the transpose (kind 1)
// or walk (kind 2) of a role group (code_off = the group's index).
enum : uint32_t { TASK_SEGMENT = 0, TASK_TRANSPOSE = 1, TASK_WALK = 2 };

struct Seg {
    uint32_t code_off;   // index into code[] (segments) or rgroups[] (role groups)
    uint32_t code_len;
    uint32_t out_slot;   // NO_SLOT if none
    uint32_t hyp;        // NO_HYP if not a hypothesis root
    uint32_t dep_off;    // index into deps[]
    uint32_t dep_cnt;
    uint32_t filler;     // filler ref of its role leaf (staged plans hold at most one), or NO_FILLER
    uint32_t kind;       // TASK_*
};

// Up to 64 role restrictions of one role, direction and role depth,
// evaluated together: the transpose turns the fillers into `parts` words per
// individual (bit s of word p = slice 32p + s's filler), the walk adds those
// words over each individual's successors in bit-sliced 3-bit saturating
// counters and maps the counts through a truth table per word.
constexpr uint32_t SLICES = 32;      // slices per FT word
constexpr uint32_t MAX_PARTS = 2;    // FT words per individual
constexpr uint32_t SLICE_MAX_N = 6;  // counting restrictions with n <= 6 can be sliced

struct RGroup {
    uint32_t role2;             // 2 * role + inverse
    uint32_t n;                 // slices in use
    uint64_t ft_off;            // byte offset of the transposed fillers (`parts` uint32 per individual)
    uint32_t parts;             // FT words per individual: 1, or MAX_PARTS when n > SLICES
    uint32_t pad;
    uint32_t want[MAX_PARTS][8];   // bit s of want[p][v]: slice 32p + s holds at count v (v = 7: 7 or more)
    uint32_t filler[SLICES * MAX_PARTS];   // filler refs (REF_NEG: count successors outside the filler)
    uint32_t out[SLICES * MAX_PARTS];      // output slots
};

struct Group {
    uint32_t item_begin;
    uint32_t seg_begin;  // index into gsegs[]
    uint32_t n_segs;
    uint32_t level;
};

// Header at the start of the workspace (plan image).
struct PlanHeader {
    uint32_t n_items, n_segs, n_groups, n_hyps;
    uint32_t n_tiles, tile_words, n_slots, flags;
    uint32_t n_levels, n_deps, n_rgroups, warp_words;   // words a warp covers per round (32, 16, 8 or 4)
    uint64_t off_segs, off_groups, off_gsegs, off_deps;
    uint64_t off_code, off_level_items, off_ctr, off_slots;
    uint64_t off_rgroups, off_ft;
    uint64_t timeout_ns;
};

// Counters region (zeroed for every execution)
struct Counters {
    uint32_t head;     // next work item
    uint32_t abort;    // set when a wait gave up
    uint32_t err;
    uint32_t pad;
    // followed by done[n_segs] (tiles finished) and acc[n_hyps][2] (TP, FP)
};

constexpr int STACK_MAX = 16;

// ------------------------------------------------------------------ host objects
struct Tuning {
    uint32_t warps = 8;
    uint32_t wpl = 1;        // words per lane
    uint32_t rounds = 2;
    uint32_t ctas_per_sm = 0;
    uint32_t timeout_ms = 2000;
    uint32_t stage = 0;      // stage role fillers in shared memory when a row fits
    uint32_t role_block = 4; // 32-edge chunks per step of the role walk (4 or 8)
    uint32_t full_occupancy = 0;  // 8-warp CTAs compiled for 8 CTAs per SM (<= 32 registers)
    uint32_t tile_words() const { return warps * 32u * wpl * rounds; }
};

constexpr size_t SMEM_OPTIN_DEFAULT = 232448;   // bytes of shared memory a CTA may opt into
constexpr int PLAN_ONLY_SMS = 152;               // planning-only handles plan for a 152-SM GB300

// Leaf rows (concept rows and slots) a warp loads ahead at the start of each
// round of a segment, in code order.
constexpr int PF_SLOTS = 8;

// Shared-memory bytes of the interpreter's stacks and leaf tables (per CTA).
inline size_t stack_smem_bytes(const Tuning &t) {
    return sizeof(uint32_t) * (size_t)t.warps * STACK_MAX * t.wpl * 32 + sizeof(uint64_t) * (size_t)t.warps * PF_SLOTS;
}

struct PlanImpl;

}  // namespace hedl

struct hedl_kb {
    uint32_t n = 0, w = 0, wp = 0;
    uint32_t n_concepts = 0, n_roles = 0, n_props = 0, n_num = 0;
    const uint32_t *concepts = nullptr;
    const float *props = nullptr;
    uint64_t prop_stride = 0;
    std::vector<hedl::DevCSR> csr_host;     // [2R]
    std::vector<uint32_t> role_edges;       // [R] forward edge counts
    hedl::DevCSR *csr_dev = nullptr;
    std::vector<hedl::DevNum> num_host;     // [Q] numeric concrete roles
    hedl::DevNum *num_dev = nullptr;
    uint32_t n_str = 0, n_strings = 0, n_str_chars = 0, n_patterns = 0;
    std::vector<hedl::DevStr> str_host;     // [S] string concrete roles
    hedl::DevStr *str_dev = nullptr;
    const uint32_t *str_off = nullptr;      // borrowed string table
    const uint8_t *str_chars = nullptr;
    uint32_t *pat_off_dev = nullptr;        // owned: pattern offsets [P+1]
    uint8_t *pat_chars_dev = nullptr;       // owned: pattern bytes
    uint32_t *contain_dev = nullptr;        // owned: [P][contain_words]
    uint64_t contain_words = 0;
    uint32_t *status_dev = nullptr;         // [4]: status, |P|, |N|, scratch
    const uint32_t *pos = nullptr, *neg = nullptr;
    uint32_t n_pos = 0, n_neg = 0;
    bool has_examples = false;
    int device = 0;
    int n_sms = 0;
    bool plan_only = false;                 // sizes only, no device state
    size_t smem_optin = hedl::SMEM_OPTIN_DEFAULT;
    void *capture_stream = nullptr;         // private stream that CUDA graphs are captured on
    hedl::Tuning tuning;
    // one cached plan for the one-shot calls
    hedl_plan *cached = nullptr;
    uint64_t cached_hash = 0;
    unsigned cached_flags = 0;
    std::vector<uint64_t> cached_progs;     // the cached plan's programs, compared on a hash match
    std::vector<uint32_t> cached_offs;
    hedl::KBView view() const;
    // a plan can name a concrete role only if the KB has one
    bool has_concrete() const { return !num_host.empty() || !str_host.empty(); }
};

struct hedl_plan {
    hedl::PlanImpl *impl = nullptr;
};

namespace hedl {

void set_error(const std::string &msg);
// Surrogate dense layer on tcgen05 tensor cores (umma.cu): C[M][N] =
// act(A[M][K] . B[N][K]^T + bias), A and B bf16 K-major, N % 256 == 0,
// K % 64 == 0, 16-byte aligned rows; *err (device, may be null) gets bit 0
// set if an MMA completion wait timed out.
struct UmmaArgs {
    const void *A;   // bf16 [M][lda]
    const void *B;   // bf16 [N][ldb]
    void *C;         // bf16 or float [M][ldc]
    const float *bias;
    int M, N, K, lda, ldb, ldc;
    int relu, out_bf16;
    uint32_t *err;
    const void *mask;   // bf16 [M][ldc] or null: outputs where mask <= 0 become 0
    // Optional fused output layer (the surrogate's N = 2 head): with w3 (bf16
    // [2][N]) set, each row's bf16-rounded outputs are also dotted with both
    // rows of w3 and the two partial sums added atomically to y (float
    // [M][2], zeroed by the caller); store = 0 then skips writing C.
    const void *w3 = nullptr;
    float *y = nullptr;
    int store = 1;
};
bool umma_shape_ok(const UmmaArgs &a);
int umma_gemm(const UmmaArgs &a, void *stream);

int fail(int code, const std::string &msg);
int cuda_fail(int cuda_err, const char *what);

// plan.cpp
struct PlanImpl {
    unsigned flags = 0;
    uint32_t n_hyps = 0;
    hedl_plan_info info{};
    std::vector<uint8_t> image;          // header + tables + zeroed counters
    void *dev_image = nullptr;           // or: the image in device memory (device-built plans), owned
    uint64_t image_bytes = 0;            // bytes to upload (aligned)
    uint64_t ctr_off = 0, ctr_bytes = 0; // counters region inside the image
    uint64_t slots_off = 0;              // slots region (after the image)
    uint64_t ws_bytes = 0;
    std::vector<uint32_t> level_items;   // [n_levels+1] item range per level
    uint32_t max_stack = 0;
    Tuning tuning;
    int bps = 0;                         // resident CTAs per SM of the interpreter
    bool staged = false;                 // role fillers staged in shared memory (one role leaf per segment)
    uint32_t n_rgroups = 0;              // bit-sliced role groups
    // plain path: validated programs
    std::vector<uint64_t> progs;
    std::vector<uint32_t> offs;
    uint32_t plain_depth = 0;
    // graph cache (a plan is captured at its second execution: a one-shot
    // plan launches directly and pays no capture)
    uint32_t runs = 0;
    void *graph_exec = nullptr;
    void *graph_ws = nullptr;
    uint32_t *graph_counts = nullptr;
    uint32_t *graph_out = nullptr;
    ~PlanImpl();
};

int validate_program(const hedl_kb *kb, const uint64_t *prog, uint32_t len, std::string *why);

}  // namespace hedl

// api.cu: shared by the entry points (C++ linkage)
int execute(hedl_kb *kb, const hedl::PlanImpl *pc, uint32_t *counts, uint32_t *out_bits, void *ws, size_t ws_bytes,
            hedl_stream s, bool upload);
int cached_plan(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, unsigned flags,
                const hedl::PlanImpl **out);

namespace hedl {
int build_plan(const hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H,
               unsigned flags, PlanImpl **out);
uint64_t hash_programs(const uint64_t *progs, const uint32_t *offs, uint32_t H);

// exec.cu / plain.cu / kb.cu launchers (return cudaError_t as int)
int launch_exec(const hedl_kb *kb, const PlanImpl *p, uint32_t *counts, uint32_t *out_bits, void *ws,
                void *stream);
// Whether plans for this KB and launch shape stage role fillers in shared memory.
bool use_staging(const hedl_kb *kb, const Tuning &t);
int launch_plain(const hedl_kb *kb, const PlanImpl *p, uint32_t *counts, uint32_t *out_bits, void *ws,
                 void *stream);
int exec_occupancy(const hedl_kb *kb, const Tuning &t, bool groups, int *blocks_per_sm);
int kb_validate_device(const hedl_kb *kb, void *stream, std::string *why);
int contain_bitmap_device(const hedl_kb *kb, void *stream);
int examples_count_device(const hedl_kb *kb, void *stream, uint32_t *np, uint32_t *nn);
size_t exec_smem_bytes(const Tuning &t);

}  // namespace hedl
