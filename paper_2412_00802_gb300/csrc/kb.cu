// Device-side checks run once when a knowledge base is registered (concept
// tails, role CSRs and their transposes, numeric- and string-role row
// pointers, string ids, the string table's offsets), the pattern-containment
// bitmap of the string table, and the example-set popcounts.  Each check ORs a bit into a flag word; nothing traps.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "device_common.cuh"

namespace hedl {

namespace {

enum : uint32_t {
    F_CONCEPT_TAIL = 1u << 0,
    F_RP_ENDS = 1u << 1,
    F_RP_ORDER = 1u << 2,
    F_COL_RANGE = 1u << 3,
    F_COL_ORDER = 1u << 4,
    F_NOT_TRANSPOSE = 1u << 5,
    F_EDGE_COUNT = 1u << 6,
    F_EXAMPLE_TAIL = 1u << 7,
    F_NUM_RP = 1u << 8,
    F_STR_RP = 1u << 9,
    F_STR_ID = 1u << 10,
    F_STR_TABLE = 1u << 11,
};

// Bits of individuals >= n and the padding words must be zero.
__global__ void concept_tail_kernel(const uint32_t *bits, uint32_t rows, uint32_t n_words, uint32_t wp, uint32_t n,
                                    uint32_t *flag) {
    const uint32_t pad = wp - n_words + 1;  // last valid word + padding words
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < (uint64_t)rows * pad;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(t / pad), k = (uint32_t)(t % pad);
        const uint32_t w = n_words - 1 + k;
        if (bits[(uint64_t)r * wp + w] & ~tail_mask(w, n_words, n)) atomicOr(flag, F_CONCEPT_TAIL);
    }
}

// A CSR is well formed: row_ptr[0] = 0, row_ptr[n] = E, rows non-decreasing,
// every row strictly increasing with ids < n.
__global__ void csr_kernel(DevCSR g, uint32_t n, uint32_t *flag) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (g.rp[0] != 0 || g.rp[n] != g.n_edges) atomicOr(flag, F_RP_ENDS);
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t lo = g.rp[i], hi = g.rp[i + 1];
        if (hi < lo || hi > g.n_edges) {
            atomicOr(flag, F_RP_ORDER);
            continue;
        }
        uint32_t prev = 0;
        for (uint32_t k = lo; k < hi; ++k) {
            const uint32_t c = g.col[k];
            if (c >= n) atomicOr(flag, F_COL_RANGE);
            if (k > lo && c <= prev) atomicOr(flag, F_COL_ORDER);
            prev = c;
        }
    }
}

// Offsets over n rows into m entries (a numeric or string role's row_ptr, the
// string table's offsets): start at 0, end at m, never decrease.
__global__ void offsets_kernel(const uint32_t *rp, uint32_t m, uint32_t n, uint32_t *flag, uint32_t bit) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (rp[0] != 0 || rp[n] != m) atomicOr(flag, bit);
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (rp[i + 1] < rp[i]) atomicOr(flag, bit);
}

// Every string id of a string role names a table string.
__global__ void str_ids_kernel(const uint32_t *ids, uint32_t m, uint32_t n_strings, uint32_t *flag) {
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x)
        if (ids[k] >= n_strings) atomicOr(flag, F_STR_ID);
}

// Bit i of row k: table string i contains pattern k (strContain of
// Algorithms 13-14, a naive scan; the empty pattern is in every string).  One
// warp per (pattern, 32 strings), a lane per string.
__global__ void contain_kernel(const uint32_t *off, const uint8_t *chars, uint32_t n_strings, const uint32_t *poff,
                               const uint8_t *pchars, uint32_t n_patterns, uint64_t words, uint32_t *out) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < (uint64_t)n_patterns * words;
         t += warps) {
        const uint32_t k = (uint32_t)(t / words);
        const uint64_t w = t % words, i = w * 32u + lane;
        bool hit = false;
        if (i < n_strings) {
            const uint32_t s0 = off[i], ls = off[i + 1] - s0, p0 = poff[k], lp = poff[k + 1] - p0;
            for (uint32_t a = 0; a + lp <= ls && !hit; ++a) {
                uint32_t j = 0;
                while (j < lp && chars[s0 + a + j] == pchars[p0 + j]) ++j;
                hit = j == lp;
            }
        }
        const uint32_t word = __ballot_sync(FULL, hit);
        if (lane == 0) out[(uint64_t)k * words + w] = word;
    }
}

// Every forward edge (a, b) appears as a in the inverse row of b.  With equal
// edge counts and both sides duplicate-free, that makes the inverse exactly
// the transpose.
__global__ void transpose_kernel(DevCSR f, DevCSR t, uint32_t n, uint32_t *flag) {
    for (uint32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const uint32_t lo = f.rp[a], hi = f.rp[a + 1];
        if (hi < lo || hi > f.n_edges) continue;  // reported by csr_kernel; never read past col
        for (uint32_t k = lo; k < hi; ++k) {
            const uint32_t b = f.col[k];
            if (b >= n) continue;  // reported by csr_kernel
            uint32_t l = t.rp[b], r = t.rp[b + 1];
            if (r < l || r > t.n_edges) {
                atomicOr(flag, F_NOT_TRANSPOSE);
                continue;
            }
            bool found = false;
            while (l < r) {
                const uint32_t m = (l + r) >> 1;
                const uint32_t c = t.col[m];
                if (c == a) {
                    found = true;
                    break;
                }
                if (c < a) l = m + 1;
                else r = m;
            }
            if (!found) atomicOr(flag, F_NOT_TRANSPOSE);
        }
    }
}

__global__ void popc_kernel(const uint32_t *a, const uint32_t *b, uint32_t n_words, uint32_t wp, uint32_t n,
                            uint32_t *out /*[2]*/, uint32_t *flag) {
    uint32_t ca = 0, cb = 0;
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < wp; w += gridDim.x * blockDim.x) {
        const uint32_t m = tail_mask(w, n_words, n);
        const uint32_t x = a[w], y = b[w];
        if ((x | y) & ~m) atomicOr(flag, F_EXAMPLE_TAIL);
        ca += __popc(x & m);
        cb += __popc(y & m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ca += __shfl_xor_sync(FULL, ca, o);
        cb += __shfl_xor_sync(FULL, cb, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        atomicAdd(out, ca);
        atomicAdd(out + 1, cb);
    }
}

std::string describe(uint32_t f) {
    std::string s;
    auto add = [&](uint32_t bit, const char *m) {
        if (f & bit) s += (s.empty() ? "" : "; ") + std::string(m);
    };
    add(F_CONCEPT_TAIL, "a concept row has bits set beyond n or in its padding words");
    add(F_RP_ENDS, "a row_ptr does not start at 0 or end at n_edges");
    add(F_RP_ORDER, "a row_ptr decreases or exceeds n_edges");
    add(F_COL_RANGE, "a CSR column id is >= n");
    add(F_COL_ORDER, "a CSR row is not strictly increasing (unsorted or duplicate assertion)");
    add(F_NOT_TRANSPOSE, "an inverse CSR is not the transpose of its forward CSR");
    add(F_EDGE_COUNT, "an inverse CSR has a different edge count than its forward CSR");
    add(F_EXAMPLE_TAIL, "an example bitset has bits set beyond n or in its padding words");
    add(F_NUM_RP, "a numeric role's row_ptr does not start at 0, decreases, or does not end at n_vals");
    add(F_STR_RP, "a string role's row_ptr does not start at 0, decreases, or does not end at n_vals");
    add(F_STR_ID, "a string role holds an id >= n_strings");
    add(F_STR_TABLE, "str_off does not start at 0, decreases, or does not end at n_str_chars");
    return s;
}

uint32_t blocks_for(uint64_t units, int n_sms) {
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((units + 255) / 256, (uint64_t)n_sms * 16));
}

}  // namespace

int kb_validate_device(const hedl_kb *kb, void *stream, std::string *why) {
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *flag = kb->status_dev + 3;
    cudaError_t e = cudaMemsetAsync(flag, 0, 4, s);
    if (e) return e;
    if (kb->n_concepts)
        concept_tail_kernel<<<blocks_for((uint64_t)kb->n_concepts * (kb->wp - kb->w + 1), kb->n_sms), 256, 0, s>>>(
            kb->concepts, kb->n_concepts, kb->w, kb->wp, kb->n, flag);
    uint32_t host_flag = 0;
    for (uint32_t r = 0; r < kb->n_roles; ++r) {
        const DevCSR &f = kb->csr_host[2 * r], &t = kb->csr_host[2 * r + 1];
        if (f.n_edges != t.n_edges) host_flag |= F_EDGE_COUNT;
        csr_kernel<<<blocks_for(kb->n, kb->n_sms), 256, 0, s>>>(f, kb->n, flag);
        csr_kernel<<<blocks_for(kb->n, kb->n_sms), 256, 0, s>>>(t, kb->n, flag);
        transpose_kernel<<<blocks_for(kb->n, kb->n_sms), 256, 0, s>>>(f, t, kb->n, flag);
    }
    for (uint32_t q = 0; q < kb->n_num; ++q)
        offsets_kernel<<<blocks_for(kb->n, kb->n_sms), 256, 0, s>>>(kb->num_host[q].rp, kb->num_host[q].n_vals,
                                                                     kb->n, flag, F_NUM_RP);
    if (kb->n_strings)
        offsets_kernel<<<blocks_for(kb->n_strings, kb->n_sms), 256, 0, s>>>(kb->str_off, kb->n_str_chars,
                                                                             kb->n_strings, flag, F_STR_TABLE);
    for (uint32_t q = 0; q < kb->n_str; ++q) {
        const DevStr &g = kb->str_host[q];
        offsets_kernel<<<blocks_for(kb->n, kb->n_sms), 256, 0, s>>>(g.rp, g.n_vals, kb->n, flag, F_STR_RP);
        if (g.n_vals)
            str_ids_kernel<<<blocks_for(g.n_vals, kb->n_sms), 256, 0, s>>>(g.ids, g.n_vals, kb->n_strings, flag);
    }
    e = cudaGetLastError();
    if (e) return e;
    uint32_t dev_flag = 0;
    e = cudaMemcpyAsync(&dev_flag, flag, 4, cudaMemcpyDeviceToHost, s);
    if (e) return e;
    e = cudaStreamSynchronize(s);
    if (e) return e;
    *why = describe(dev_flag | host_flag);
    return 0;
}

int contain_bitmap_device(const hedl_kb *kb, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!kb->contain_words || !kb->n_patterns) return 0;
    const uint64_t warps = (uint64_t)kb->n_patterns * kb->contain_words;
    contain_kernel<<<blocks_for(warps * 32u, kb->n_sms), 256, 0, s>>>(kb->str_off, kb->str_chars, kb->n_strings,
                                                                      kb->pat_off_dev, kb->pat_chars_dev,
                                                                      kb->n_patterns, kb->contain_words,
                                                                      kb->contain_dev);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    return cudaStreamSynchronize(s);
}

int examples_count_device(const hedl_kb *kb, void *stream, uint32_t *np, uint32_t *nn) {
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *cnt = kb->status_dev + 4;   // [2]
    uint32_t *flag = kb->status_dev + 3;
    cudaError_t e = cudaMemsetAsync(kb->status_dev + 3, 0, 12, s);
    if (e) return e;
    popc_kernel<<<blocks_for(kb->wp, kb->n_sms), 256, 0, s>>>(kb->pos, kb->neg, kb->w, kb->wp, kb->n, cnt, flag);
    e = cudaGetLastError();
    if (e) return e;
    uint32_t h[3];
    e = cudaMemcpyAsync(h, kb->status_dev + 3, 12, cudaMemcpyDeviceToHost, s);
    if (e) return e;
    e = cudaStreamSynchronize(s);
    if (e) return e;
    if (h[0]) return -1;
    *np = h[1];
    *nn = h[2];
    return 0;
}

}  // namespace hedl
