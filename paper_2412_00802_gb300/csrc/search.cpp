// Canonical form of hypothesis programs for the refinement search: every
// AND / OR gets its two operands in ascending order of their canonical
// instruction bytes, so commuted duplicates of a candidate collapse to one
// program before they are scored.  Host code; the paper's engine evaluates
// hypotheses one by one and has no counterpart.
#include <cstring>
#include <string>
#include <vector>

#include "hedl_internal.h"

namespace hedl {
namespace {

int arity(uint32_t op) {
    if (op == HEDL_OP_NOT || (op >= HEDL_OP_EXISTS && op <= HEDL_OP_EXACTLY)) return 1;
    if (op == HEDL_OP_AND || op == HEDL_OP_OR) return 2;
    if (op >= HEDL_OP_ATOM && op <= HEDL_OP_SCONTAINS) return 0;
    return -1;
}

// a < b as byte strings of little-endian words (a proper prefix is smaller)
bool bytes_less(const uint64_t *a, size_t la, const uint64_t *b, size_t lb) {
    const int c = std::memcmp(a, b, 8 * (la < lb ? la : lb));
    return c < 0 || (c == 0 && la < lb);
}

}  // namespace
}  // namespace hedl

using namespace hedl;

extern "C" int hedl_canonical_batch(const uint64_t *progs, const uint32_t *offs, uint32_t H, uint64_t *out) {
    if (!offs || (H && offs[H] && (!progs || !out))) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    struct Span {
        uint32_t start, len;
    };
    std::vector<Span> st;
    std::vector<uint64_t> tmp;
    for (uint32_t h = 0; h < H; ++h) {
        const uint32_t o0 = offs[h], L = offs[h + 1] - offs[h];
        if (offs[h + 1] < o0) return fail(HEDL_ERR_INVALID_ARG, "offsets decrease at program " + std::to_string(h));
        uint64_t *dst = out + o0;
        st.clear();
        for (uint32_t k = 0; k < L; ++k) {
            const uint64_t w = progs[o0 + k];
            const int a = arity((uint32_t)(w & 0xFF));
            if (a < 0 || (int)st.size() < a)
                return fail(HEDL_ERR_BAD_PROGRAM, "program " + std::to_string(h) + ": not a valid postfix program");
            dst[k] = w;   // children occupy dst[k - their lengths .. k)
            if (a == 0) {
                st.push_back({k, 1});
            } else if (a == 1) {
                Span c = st.back();
                st.back() = {c.start, c.len + 1};
            } else {
                const Span y = st.back();
                st.pop_back();
                const Span x = st.back();
                if (bytes_less(dst + y.start, y.len, dst + x.start, x.len)) {   // operands swap places
                    tmp.assign(dst + x.start, dst + x.start + x.len);
                    std::memmove(dst + x.start, dst + y.start, 8ull * y.len);
                    std::memcpy(dst + x.start + y.len, tmp.data(), 8ull * x.len);
                }
                st.back() = {x.start, x.len + y.len + 1};
            }
        }
        if (st.size() != 1)
            return fail(HEDL_ERR_BAD_PROGRAM, "program " + std::to_string(h) + ": not a valid postfix program");
    }
    return HEDL_OK;
}
