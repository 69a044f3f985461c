// Device building blocks shared by the batched interpreter (exec.cu) and the
// one-operation-per-launch path (plain.cu).
//
// Layout: a set of individuals is a row of uint32 words, bit i of word w =
// individual 32*w + i.  A warp works on 32*WPL consecutive words; lane l holds
// words wb + l*WPL .. wb + l*WPL + WPL-1 (so WPL = 4 gives 128-bit loads).
#pragma once

#include <cstdint>

#include "hedl_internal.h"

namespace hedl {

constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t tail_mask(uint32_t w, uint32_t n_words, uint32_t n) {
    if (w + 1 < n_words) return FULL;
    if (w + 1 == n_words) {
        uint32_t r = n & 31u;
        return r ? ((1u << r) - 1u) : FULL;
    }
    return 0u;
}

// bits lo..hi-1 set (0 <= lo <= hi <= 32)
__device__ __forceinline__ uint32_t range_mask(uint32_t lo, uint32_t hi) {
    uint32_t up = hi >= 32 ? FULL : ((1u << hi) - 1u);
    uint32_t dn = lo >= 32 ? FULL : ((1u << lo) - 1u);
    return up & ~dn;
}

template <int WPL>
__device__ __forceinline__ void load_row_ro(const uint32_t *__restrict__ row, uint32_t wb, uint32_t lane,
                                            uint32_t wp, uint32_t (&v)[WPL]) {
    uint32_t w0 = wb + lane * WPL;
    if constexpr (WPL == 4) {
        if (w0 < wp) {
            uint4 q = __ldg(reinterpret_cast<const uint4 *>(row + w0));
            v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
        } else {
            v[0] = v[1] = v[2] = v[3] = 0u;
        }
    } else {
#pragma unroll
        for (int s = 0; s < WPL; ++s) v[s] = (w0 + s < wp) ? __ldg(row + w0 + s) : 0u;
    }
}

// Rows written earlier in the same kernel (slots) are read with plain loads,
// never through the read-only path.
template <int WPL>
__device__ __forceinline__ void load_row_rw(const uint32_t *row, uint32_t wb, uint32_t lane, uint32_t wp,
                                            uint32_t (&v)[WPL]) {
    uint32_t w0 = wb + lane * WPL;
    if constexpr (WPL == 4) {
        if (w0 < wp) {
            uint4 q = *reinterpret_cast<const uint4 *>(row + w0);
            v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
        } else {
            v[0] = v[1] = v[2] = v[3] = 0u;
        }
    } else {
#pragma unroll
        for (int s = 0; s < WPL; ++s) v[s] = (w0 + s < wp) ? row[w0 + s] : 0u;
    }
}

template <int WPL>
__device__ __forceinline__ void store_row(uint32_t *row, uint32_t wb, uint32_t lane, uint32_t wp,
                                          const uint32_t (&v)[WPL]) {
    uint32_t w0 = wb + lane * WPL;
    if constexpr (WPL == 4) {
        if (w0 < wp) *reinterpret_cast<uint4 *>(row + w0) = make_uint4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int s = 0; s < WPL; ++s)
            if (w0 + s < wp) row[w0 + s] = v[s];
    }
}

// Does count `cnt` decide the restriction?  Returns the threshold at which the
// answer can no longer change (the walk over a row may stop there).
__device__ __forceinline__ uint64_t decide_cap(uint32_t kind, uint32_t n) {
    switch (kind) {
    case HEDL_OP_EXISTS: return 1;             // one C-successor
    case HEDL_OP_FORALL: return 1;             // one successor outside C
    case HEDL_OP_ATLEAST: return n;
    default: return (uint64_t)n + 1;           // ATMOST / EXACTLY: n+1 of them
    }
}

__device__ __forceinline__ bool role_pred(uint32_t kind, uint32_t cnt, uint32_t n) {
    switch (kind) {
    case HEDL_OP_EXISTS: return cnt >= 1;
    case HEDL_OP_FORALL: return cnt == 0;      // cnt counts successors NOT in C
    case HEDL_OP_ATLEAST: return cnt >= n;
    case HEDL_OP_ATMOST: return cnt <= n;
    default: return cnt == n;                  // EXACTLY
    }
}

// Streaming read of KB arrays (CSR): read-only for the kernel's lifetime and
// used once per pass, so they do not take L1 lines from the filler bitsets.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) {
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}


// Role restriction over the warp's 32*WPL words (Algorithms 3-8 of the
// paper, recast).  For each word (32 individuals) the warp walks the word's
// CSR edge range, a block of BLK (<= 32) chunks of 32 edges at a time: lane e
// loads edge e of each chunk (coalesced), tests the filler bit of its object,
// and a ballot packs each chunk's tests into a mask that lane c keeps for
// chunk c.  A warp scan turns the masks' popcounts into prefix counts, so
// lane i counts the hits inside its own row [lo, hi) with two rank lookups,
// however many chunks the row spans.  Counts stay in registers (no atomics,
// no counter matrix), and the walk stops once every lane's answer is decided.
// FORALL counts successors outside the filler.
// filler_inverted: the caller already complemented a FORALL filler.
template <int WPL, int BLK>
__device__ __forceinline__ void role_words(const DevCSR g, const uint32_t *filler, uint32_t kind, uint32_t n_arg,
                                           uint32_t n, uint32_t n_words, uint32_t wb, uint32_t lane,
                                           uint32_t (&v)[WPL], bool filler_inverted = false) {
    static_assert(BLK >= 1 && BLK <= 32, "a block holds 1..32 chunks");
    constexpr int ROLE_BLOCK = BLK;
    constexpr uint32_t BE = 32u * ROLE_BLOCK;     // edges per block
    const uint32_t neg = (kind == HEDL_OP_FORALL && !filler_inverted) ? 1u : 0u;
    const uint64_t cap = decide_cap(kind, n_arg);
    const uint32_t *__restrict__ rp = g.rp;
    const uint32_t *__restrict__ col = g.col;
    uint32_t nlo = 0, nhi = 0;   // row pointers of the next word, fetched ahead
    {
        const uint32_t i = wb * 32u + lane;
        if (wb < n_words && i < n) {
            nlo = ld_stream(rp + i);
            nhi = ld_stream(rp + i + 1);
        }
    }
#pragma unroll 1
    for (int j = 0; j < 32; ++j) {
#pragma unroll
        for (int s = 0; s < WPL; ++s) {
            const uint32_t w = wb + (uint32_t)j * WPL + s;
            uint32_t word = 0;
            if (w < n_words) {
                const uint32_t i = w * 32u + lane;
                const bool valid = i < n;
                const uint32_t lo = nlo, hi = nhi;
                {
                    const uint32_t i2 = i + 32u;
                    if (w + 1 < n_words && i2 < n) {
                        nlo = ld_stream(rp + i2);
                        nhi = ld_stream(rp + i2 + 1);
                    }
                }
                const uint32_t nv = min(32u, n - w * 32u);
                const uint32_t e0 = __shfl_sync(FULL, lo, 0);
                const uint32_t e1 = __shfl_sync(FULL, hi, nv - 1);
                // my row relative to the word's first edge (empty for lanes past n)
                const uint32_t r0 = valid ? lo - e0 : 0u, r1 = valid ? hi - e0 : 0u;
                uint32_t cnt = 0;
                if (cap > 0) {
#pragma unroll 1
                    for (uint32_t rb = 0; rb < e1 - e0; rb += BE) {
                        const uint32_t base = e0 + rb;
                        // Edge index clamped to the word's last edge: lanes past the end reload
                        // a valid edge, and their bits lie beyond every row so no rank counts them.
                        uint32_t hit[ROLE_BLOCK];
#pragma unroll
                        for (int u = 0; u < ROLE_BLOCK; ++u)
                            hit[u] = ld_stream(col + min(base + 32u * u + lane, e1 - 1u));
#pragma unroll
                        for (int u = 0; u < ROLE_BLOCK; ++u)
                            hit[u] = (__funnelshift_r(filler[hit[u] >> 5], 0u, hit[u]) & 1u) ^ neg;
                        uint32_t mc = 0;   // lane c < ROLE_BLOCK: mask of chunk c
#pragma unroll
                        for (int u = 0; u < ROLE_BLOCK; ++u) {
                            const uint32_t m = __ballot_sync(FULL, hit[u]);
                            if (lane == (uint32_t)u) mc = m;
                        }
                        // exclusive prefix of the chunks' popcounts over lanes 0..ROLE_BLOCK-1
                        const uint32_t pc = __popc(mc);
                        uint32_t incl = pc;
#pragma unroll
                        for (int o = 1; o < ROLE_BLOCK; o <<= 1) {
                            const uint32_t t = __shfl_up_sync(FULL, incl, o);
                            if (lane >= (uint32_t)o) incl += t;
                        }
                        const uint32_t excl = incl - pc;
                        // hits before block-relative position x in [0, BE]
                        auto rank = [&](uint32_t x) -> uint32_t {
                            const uint32_t c = min(x >> 5, (uint32_t)ROLE_BLOCK - 1);
                            const uint32_t e = __shfl_sync(FULL, excl, c);
                            const uint32_t m = __shfl_sync(FULL, mc, c);
                            const uint32_t sh = x - 32u * c;   // 0..32
                            return e + __popc(sh >= 32u ? m : (m & ((1u << sh) - 1u)));
                        };
                        const uint32_t a = r0 > rb ? min(r0 - rb, BE) : 0u;
                        const uint32_t z = r1 > rb ? min(r1 - rb, BE) : 0u;
                        cnt += rank(z) - rank(a);
                        const bool done = !valid || r1 <= rb + BE || (uint64_t)cnt >= cap;
                        if (__all_sync(FULL, done)) break;
                    }
                }
                word = __ballot_sync(FULL, valid && role_pred(kind, cnt, n_arg));
            }
            if (lane == (uint32_t)j) v[s] = word;
        }
    }
}

// Role restriction over the warp's words as ONE edge stream (the interpreter's
// walk).  The words wb .. wb+K-1 are consecutive individuals, so their CSR
// rows form one contiguous edge range [E0, E1).  The warp reads that range in
// blocks of BLK 32-edge chunks, always loading the next block while it tests
// the current one (the gather's DRAM latency overlaps the filler lookups),
// and attributes each block's hits to the words whose rows it covers: lane i
// of word k counts the hits inside its row with two rank lookups, as in
// role_words, and a word is emitted (ballot) once its last edge has passed.
// A word whose every lane is decided (cap reached or row ended) makes the
// stream jump to the next word's first edge.  Word k of the warp goes to lane
// k / WPL, slot k % WPL.  n_words bounds the warp's words; lanes of
// individuals >= n hold empty rows and emit 0.
template <int WPL, int BLK>
__device__ __forceinline__ void role_stream(const DevCSR g, const uint32_t *filler, uint32_t kind, uint32_t n_arg,
                                            uint32_t n, uint32_t n_words, uint32_t wb, uint32_t lane,
                                            uint32_t (&v)[WPL], bool filler_inverted = false) {
    static_assert(BLK >= 1 && BLK <= 32, "a block holds 1..32 chunks");
    constexpr uint32_t BE = 32u * BLK;     // edges per block
    const uint32_t neg = (kind == HEDL_OP_FORALL && !filler_inverted) ? 1u : 0u;
    const uint64_t cap = decide_cap(kind, n_arg);
    const uint32_t *__restrict__ rp = g.rp;
    const uint32_t *__restrict__ col = g.col;
#pragma unroll
    for (int s = 0; s < WPL; ++s) v[s] = 0u;
    if (wb >= n_words) return;
    const uint32_t K = min(32u * WPL, n_words - wb);
    auto put = [&](uint32_t k, uint32_t word) {
#pragma unroll
        for (int s = 0; s < WPL; ++s)
            if (lane == k / WPL && k % WPL == (uint32_t)s) v[s] = word;
    };
    auto lane_valid = [&](uint32_t k) { return (wb + k) * 32u + lane < n; };
    if (cap == 0) {   // decided before any edge (at least 0): every individual
        for (uint32_t k = 0; k < K; ++k) put(k, __ballot_sync(FULL, lane_valid(k)));
        return;
    }
    // row pointers of words k, k+1, k+2 (empty rows for lanes past n or words past K)
    auto ld_rows = [&](uint32_t k, uint32_t &lo, uint32_t &hi) {
        const uint32_t i = (wb + k) * 32u + lane;
        if (k < K && i < n) {
            lo = ld_stream(rp + i);
            hi = ld_stream(rp + i + 1);
        } else {
            lo = 0u;
            hi = 0u;
        }
    };
    // last edge (exclusive) of word k, from its last valid lane
    auto word_end = [&](uint32_t k, uint32_t hi) {
        const uint32_t nv = min(32u, n - (wb + k) * 32u);
        return __shfl_sync(FULL, hi, nv - 1u);
    };
    uint32_t lo0, hi0, lo1, hi1, lo2, hi2;
    ld_rows(0, lo0, hi0);
    ld_rows(1, lo1, hi1);
    ld_rows(2, lo2, hi2);
    const uint32_t E0 = __shfl_sync(FULL, lo0, 0);
    const uint32_t E1 = ld_stream(rp + min(n, (wb + K) * 32u));
    uint32_t k = 0, cnt = 0;
    uint32_t ew1 = word_end(0, hi0);
    auto next_word = [&]() {
        lo0 = lo1, hi0 = hi1, lo1 = lo2, hi1 = hi2;
        ld_rows(k + 2, lo2, hi2);
        ew1 = word_end(k, hi0);
        cnt = 0;
    };
    uint32_t pf[BLK];
    auto fetch = [&](uint32_t at) {
#pragma unroll
        for (int u = 0; u < BLK; ++u) pf[u] = ld_stream(col + min(at + 32u * u + lane, E1 - 1u));
    };
    uint32_t base = E0;
    if (base < E1) fetch(base);
#pragma unroll 1
    while (base < E1) {
        uint32_t hit[BLK];
#pragma unroll
        for (int u = 0; u < BLK; ++u) hit[u] = pf[u];
        const uint32_t nb = base + BE;
        if (nb < E1) fetch(nb);
        // Positions past E1 reloaded edge E1-1; they lie beyond every row, so no rank counts them.
#pragma unroll
        for (int u = 0; u < BLK; ++u) hit[u] = (__funnelshift_r(filler[hit[u] >> 5], 0u, hit[u]) & 1u) ^ neg;
        uint32_t mc = 0;   // lane c < BLK: mask of chunk c
#pragma unroll
        for (int u = 0; u < BLK; ++u) {
            const uint32_t m = __ballot_sync(FULL, hit[u]);
            if (lane == (uint32_t)u) mc = m;
        }
        const uint32_t pc = __popc(mc);
        uint32_t incl = pc;
#pragma unroll
        for (int o = 1; o < BLK; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        const uint32_t excl = incl - pc;
        // hits before block-relative position x in [0, BE]
        auto rank = [&](uint32_t x) -> uint32_t {
            const uint32_t c = min(x >> 5, (uint32_t)BLK - 1);
            const uint32_t e = __shfl_sync(FULL, excl, c);
            const uint32_t m = __shfl_sync(FULL, mc, c);
            const uint32_t sh = x - 32u * c;   // 0..32
            return e + __popc(sh >= 32u ? m : (m & ((1u << sh) - 1u)));
        };
        // the words whose rows meet this block, in order
        bool finished = false;
#pragma unroll 1
        for (;;) {
            const uint32_t a = lo0 > base ? min(lo0 - base, BE) : 0u;
            const uint32_t z = hi0 > base ? min(hi0 - base, BE) : 0u;
            cnt += rank(z) - rank(a);
            if (ew1 > nb) break;                       // word k goes on in the next block
            put(k, __ballot_sync(FULL, lane_valid(k) && role_pred(kind, cnt, n_arg)));
            if (++k == K) {
                finished = true;
                break;
            }
            next_word();
        }
        if (finished) return;
        // word k spans past this block: skip the rest of it once every lane is decided
        const bool decided = !lane_valid(k) || hi0 <= nb || (uint64_t)cnt >= cap;
        if (__all_sync(FULL, decided)) {
            put(k, __ballot_sync(FULL, lane_valid(k) && role_pred(kind, cnt, n_arg)));
            if (++k == K) return;
            const uint32_t nxt = ew1;                  // the next word's first edge
            next_word();
            if (nxt != nb && nxt < E1) fetch(nxt);
            base = nxt;
        } else {
            base = nb;
        }
    }
    // the stream ended (or was empty): the remaining words have no edges left
    for (; k < K; ++k) {
        put(k, __ballot_sync(FULL, lane_valid(k) && role_pred(kind, cnt, n_arg)));
        cnt = 0;
    }
}

__device__ __forceinline__ bool data_cmp(uint32_t cmp, float x, float t);

// Numeric data-range restriction (Algorithms 9-10): one float compare per
// individual.  Lane l builds its own words wb + l*WPL + s from the 32
// contiguous values of each (eight 16-byte loads, all in flight at once, when
// the row is 16-byte aligned and the word is whole; scalar loads otherwise).
// NaN (missing) compares false.
template <int WPL>
__device__ __forceinline__ void data_words(const float *__restrict__ vals, uint32_t cmp, float t, uint32_t n,
                                           uint32_t n_words, uint32_t wb, uint32_t lane, uint32_t (&v)[WPL]) {
    const bool vec = (reinterpret_cast<uintptr_t>(vals) & 15u) == 0;
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
        const uint32_t w = wb + lane * WPL + s;
        uint32_t word = 0;
        if (w < n_words) {
            const uint32_t i0 = w * 32u;
            if (vec && i0 + 32u <= n) {
                float4 q[8];
                const float4 *p4 = reinterpret_cast<const float4 *>(vals + i0);
#pragma unroll
                for (int k = 0; k < 8; ++k) q[k] = __ldg(p4 + k);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    word |= (uint32_t)data_cmp(cmp, q[k].x, t) << (4 * k);
                    word |= (uint32_t)data_cmp(cmp, q[k].y, t) << (4 * k + 1);
                    word |= (uint32_t)data_cmp(cmp, q[k].z, t) << (4 * k + 2);
                    word |= (uint32_t)data_cmp(cmp, q[k].w, t) << (4 * k + 3);
                }
            } else {
                for (uint32_t k = 0; k < 32u && i0 + k < n; ++k)
                    word |= (uint32_t)data_cmp(cmp, __ldg(vals + i0 + k), t) << k;
            }
        }
        v[s] = word;
    }
}

__device__ __forceinline__ bool data_cmp(uint32_t cmp, float x, float t) {
    return cmp == HEDL_OP_DGE ? (x >= t) : cmp == HEDL_OP_DLE ? (x <= t) : (x == t);
}

// The test a concrete-role restriction applies to each asserted value (the
// 32-bit word of a float value or of a string id): a float compare (numeric
// roles, Algorithms 9-10), id equality (string EQUAL, Algorithms 11-12) or a
// bit of the pattern's containment row (string CONTAIN, Algorithms 13-14).
// ValueTest carries the kind at run time; exist_words is compiled once per
// kind (FloatTest, IdEqTest, IdBitTest) and dispatched once per restriction.
struct ValueTest {
    enum : uint32_t { FLOAT_CMP = 0, ID_EQ = 1, ID_BIT = 2 };
    uint32_t mode;
    uint32_t cmp;           // FLOAT_CMP: HEDL_OP_DGE / DLE / DEQ
    uint32_t arg;           // FLOAT_CMP: the threshold's bits; ID_EQ: the string id
    const uint32_t *bits;   // ID_BIT: the containment row
};
struct FloatTest {
    uint32_t cmp;
    float t;
    __device__ __forceinline__ bool operator()(uint32_t x) const { return data_cmp(cmp, __uint_as_float(x), t); }
};
struct IdEqTest {
    uint32_t id;
    __device__ __forceinline__ bool operator()(uint32_t x) const { return x == id; }
};
struct IdBitTest {
    const uint32_t *bits;
    __device__ __forceinline__ bool operator()(uint32_t x) const { return (__ldg(bits + (x >> 5)) >> (x & 31u)) & 1u; }
};

// Existential restriction on a concrete role with several values per
// subject (Section III-B): individual i belongs iff one of its values
// vals[rp[i] .. rp[i+1]) passes the test.  The 32 individuals of a word own
// one contiguous run of values; the warp reads it EX_STEP values a step (four
// coalesced loads), ballots the tests, and each lane tests the bits that fall
// in its own sub-range.  The words are software-pipelined: while word w is
// tested, the first steps of words w+1 and w+2 and the row pointers of words
// w+3 and w+4 are in flight (a word's first step is fetched two words after
// its row pointers), so a word whose run fits one step costs a fraction of a
// memory latency.  A longer run continues step by step and the warp
// leaves it once every individual whose values reach past the step has found
// one (the paper's skip over a subject already satisfied), so a heavy subject
// costs 1/32 of a lane walk.
constexpr uint32_t EX_LOADS = 4;
constexpr uint32_t EX_STEP = 32u * EX_LOADS;

// this lane's row of word w (empty past the warp's words or past n)
__device__ __forceinline__ void ex_row(const uint32_t *rp, uint32_t w, uint32_t n_words, uint32_t n, uint32_t lane,
                                       uint32_t &lo, uint32_t &hi) {
    lo = hi = 0;
    const uint32_t i = w * 32u + lane;
    if (w < n_words && i < n) {
        lo = ld_stream(rp + i);
        hi = ld_stream(rp + i + 1);
    }
}

// the values [c, c + EX_STEP) of a run ending at end, one per lane and load
__device__ __forceinline__ void ex_fetch(const uint32_t *vals, uint32_t c, uint32_t end, uint32_t lane,
                                         uint32_t (&x)[EX_LOADS]) {
#pragma unroll
    for (uint32_t u = 0; u < EX_LOADS; ++u) {
        const uint32_t k = c + 32u * u + lane;
        x[u] = k < end ? __ldg(vals + k) : 0u;
    }
}

// does a value in [c, c + EX_STEP) of this lane's row [lo, hi) pass?
template <class Test>
__device__ __forceinline__ bool ex_test(const uint32_t (&x)[EX_LOADS], uint32_t c, uint32_t end, uint32_t lo,
                                        uint32_t hi, uint32_t lane, const Test &test) {
    bool hit = false;
#pragma unroll
    for (uint32_t u = 0; u < EX_LOADS; ++u) {
        const uint32_t cu = c + 32u * u;
        const uint32_t m = __ballot_sync(FULL, cu + lane < end && test(x[u]));
        const uint32_t a = lo > cu ? min(lo - cu, 32u) : 0u, b = hi > cu ? min(hi - cu, 32u) : 0u;
        hit = hit || (m & range_mask(a, b)) != 0u;
    }
    return hit;
}

template <int WPL, class Test>
__device__ __forceinline__ void exist_words(const uint32_t *rp, const uint32_t *vals, const Test test, uint32_t n,
                                            uint32_t n_words, uint32_t wb, uint32_t lane, uint32_t (&v)[WPL]) {
    // rows [loK, hiK) of words w .. w+3; runs [bK, eK) and first steps xK of words w, w+1
    uint32_t lo0, hi0, lo1, hi1, lo2, hi2, lo3, hi3;
    ex_row(rp, wb, n_words, n, lane, lo0, hi0);
    ex_row(rp, wb + 1, n_words, n, lane, lo1, hi1);
    ex_row(rp, wb + 2, n_words, n, lane, lo2, hi2);
    ex_row(rp, wb + 3, n_words, n, lane, lo3, hi3);
    uint32_t b0 = __shfl_sync(FULL, lo0, 0), e0 = __reduce_max_sync(FULL, hi0);
    uint32_t b1 = __shfl_sync(FULL, lo1, 0), e1 = __reduce_max_sync(FULL, hi1);
    uint32_t x0[EX_LOADS], x1[EX_LOADS];
    ex_fetch(vals, b0, e0, lane, x0);
    ex_fetch(vals, b1, e1, lane, x1);
    for (int j = 0; j < 32; ++j) {
#pragma unroll
        for (int s = 0; s < WPL; ++s) {
            const uint32_t w = wb + (uint32_t)j * WPL + s;   // the words go in order: w + 1 is the next
            uint32_t word = 0;
            if (w < n_words) {   // warp-uniform; then lane 0's individual 32w < n exists
                // start word w+2's first step (its rows came two words ago) and word w+4's rows
                const uint32_t b2 = __shfl_sync(FULL, lo2, 0), e2 = __reduce_max_sync(FULL, hi2);
                uint32_t x2[EX_LOADS];
                ex_fetch(vals, b2, e2, lane, x2);
                uint32_t lo4, hi4;
                ex_row(rp, w + 4, n_words, n, lane, lo4, hi4);
                // test word w
                bool hit = ex_test(x0, b0, e0, lo0, hi0, lane, test);
                for (uint32_t c = b0 + EX_STEP; c < e0; c += EX_STEP) {
                    if (__all_sync(FULL, hit || hi0 <= c)) break;
                    uint32_t y[EX_LOADS];
                    ex_fetch(vals, c, e0, lane, y);
                    hit = ex_test(y, c, e0, lo0, hi0, lane, test) || hit;
                }
                word = __ballot_sync(FULL, hit);
                lo0 = lo1, hi0 = hi1, b0 = b1, e0 = e1;
                lo1 = lo2, hi1 = hi2, b1 = b2, e1 = e2;
                lo2 = lo3, hi2 = hi3;
                lo3 = lo4, hi3 = hi4;
#pragma unroll
                for (uint32_t u = 0; u < EX_LOADS; ++u) {
                    x0[u] = x1[u];
                    x1[u] = x2[u];
                }
            }
            if (lane == (uint32_t)j) v[s] = word;
        }
    }
}

// exist_words with the test's kind resolved at compile time (one dispatch per
// restriction, warp-uniform).
template <int WPL>
__device__ __forceinline__ void exist_words(const uint32_t *rp, const uint32_t *vals, const ValueTest &test,
                                            uint32_t n, uint32_t n_words, uint32_t wb, uint32_t lane,
                                            uint32_t (&v)[WPL]) {
    if (test.mode == ValueTest::FLOAT_CMP)
        exist_words<WPL>(rp, vals, FloatTest{test.cmp, __uint_as_float(test.arg)}, n, n_words, wb, lane, v);
    else if (test.mode == ValueTest::ID_EQ)
        exist_words<WPL>(rp, vals, IdEqTest{test.arg}, n, n_words, wb, lane, v);
    else
        exist_words<WPL>(rp, vals, IdBitTest{test.bits}, n, n_words, wb, lane, v);
}

// The test of a D_DATA instruction on a numeric or string role (op word bit 8
// or 9; aux = the op; b = threshold bits, string id or pattern id).
__host__ __device__ __forceinline__ ValueTest value_test(const KBView &kb, uint32_t op_word, uint32_t b) {
    const uint32_t op = (op_word >> 16) & 0xFFu;
    if (op == HEDL_OP_SEQ) return ValueTest{ValueTest::ID_EQ, 0u, b, nullptr};
    if (op == HEDL_OP_SCONTAINS) return ValueTest{ValueTest::ID_BIT, 0u, 0u, kb.contain + (uint64_t)b * kb.contain_words};
    return ValueTest{ValueTest::FLOAT_CMP, op, b, nullptr};
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace hedl
