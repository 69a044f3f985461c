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

// A hint to bring bytes [p, p + bytes) into L2 (p 16-byte aligned, bytes a
// multiple of 16, the range inside one allocation); no register waits on it.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L2 prefetch of a[lo, hi) by lane 0 (a 16-byte aligned): the start is
// rounded down and the size down to whole 16-byte units, so the hint stays
// inside [0, hi).
__device__ __forceinline__ void prefetch_range(const uint32_t *a, uint32_t lo, uint32_t hi, uint32_t lane) {
    if (lane != 0u || lo >= hi) return;
    lo &= ~3u;
    const uint32_t bytes = ((hi - lo) * 4u) & ~15u;
    if (bytes) prefetch_l2(a + lo, bytes);
}

// the same for four consecutive words (p 16-byte aligned)
__device__ __forceinline__ uint4 ld_stream4(const uint32_t *p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
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
// the current one (the gather's DRAM latency overlaps the filler lookups) and
// asking L2 for the blocks after it (prefetch hints that hold no registers),
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
    // L2 hints (no registers held): the warp's row pointers, and the edge
    // blocks two to four ahead of the one loading into registers
    const bool cvec = (reinterpret_cast<uintptr_t>(col) & 15u) == 0;
    if ((reinterpret_cast<uintptr_t>(rp) & 15u) == 0) prefetch_range(rp, wb * 32u, min(n, (wb + K) * 32u) + 1u, lane);
    auto ahead = [&](uint32_t from, uint32_t blocks) {
        if (cvec && from < E1) prefetch_range(col, from, min(E1, from + blocks * BE), lane);
    };
    uint32_t base = E0;
    if (base < E1) fetch(base);
    ahead(E0 + BE, 3u);
#pragma unroll 1
    while (base < E1) {
        uint32_t hit[BLK];
#pragma unroll
        for (int u = 0; u < BLK; ++u) hit[u] = pf[u];
        const uint32_t nb = base + BE;
        if (nb < E1) fetch(nb);
        ahead(base + 4u * BE, 1u);
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
            if (nxt != nb && nxt < E1) {
                fetch(nxt);
                ahead(nxt + BE, 3u);
            }
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
// kind (each float compare, IdEqTest, IdBitTest) and dispatched once per
// restriction.
struct ValueTest {
    enum : uint32_t { FLOAT_CMP = 0, ID_EQ = 1, ID_BIT = 2 };
    uint32_t mode;
    uint32_t cmp;           // FLOAT_CMP: HEDL_OP_DGE / DLE / DEQ
    uint32_t arg;           // FLOAT_CMP: the threshold's bits; ID_EQ: the string id
    const uint32_t *bits;   // ID_BIT: the containment row
};
template <uint32_t CMP>
struct FloatTest {
    float t;
    __device__ __forceinline__ bool operator()(uint32_t x) const {
        const float f = __uint_as_float(x);
        return CMP == HEDL_OP_DGE ? (f >= t) : CMP == HEDL_OP_DLE ? (f <= t) : (f == t);
    }
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
// vals[rp[i] .. rp[i+1]) passes the test.  The warp's 32*WPL words are
// 1024*WPL consecutive individuals, so their values form one contiguous run,
// and the warp streams that run once, in windows of EX_WIN values.  Each lane
// loads four 16-byte vectors of a window (each load coalesced over 512
// bytes), and the warp turns the tests into the window's 512-bit pass mask:
// lane k < 16 keeps mask word k and the position of the first pass in the
// words after it.  The row pointers come four words at a time (lane l loads
// rp[32w + l] of each, the next four in flight), and each lane finds the
// first pass at or after its row's start with two shuffles and compares it
// with the row's end.  The next window's values are in flight while the
// current one is looked up, and the warp's row pointers are requested into L2
// when it starts (a bulk prefetch hint, which holds no registers).  Hinting
// the values too was slower where several restrictions read one role's
// values at once.  A window is loaded only while a row that has
// not passed yet reaches into it, and the stream jumps straight to the first
// such row, so a subject already satisfied is skipped (the paper's early
// exit): a heavy subject costs its values up to the window of its first
// pass.  Value counts stay below 2^31 (the KB loader's limit), so positions
// relative to a window fit signed 32-bit arithmetic.
constexpr uint32_t EX_LOADS = 4;               // 16-byte loads per lane per window
constexpr uint32_t EX_WIN = 128u * EX_LOADS;   // values per window
constexpr uint32_t EX_NONE = 0x7FFFFFFFu;      // no pass

// The row pointers of words w0 .. w0+3: r[q] = rp[32(w0 + q) + lane],
// tail = rp[32 w0 + 128], zero past n (a zero end makes a row empty).
struct ExRows {
    uint32_t r[4];
    uint32_t tail;
};
__device__ __forceinline__ void ex_rows(ExRows &b, const uint32_t *rp, uint32_t w0, uint32_t w_end, uint32_t n,
                                        uint32_t lane) {
    if (w0 >= w_end) return;   // warp-uniform; nothing reads this batch
#pragma unroll
    for (uint32_t q = 0; q < 4u; ++q) {
        const uint32_t i = 32u * (w0 + q) + lane;
        b.r[q] = i <= n ? ld_stream(rp + i) : 0u;
    }
    const uint32_t t = 32u * w0 + 128u;
    b.tail = t <= n ? ld_stream(rp + t) : 0u;
}

// the window [c, c + EX_WIN) of a run ending at end (c a multiple of 128):
// lane l's vector u holds values c + 128u + 4l .. + 3 (zero at and past end)
__device__ __forceinline__ void ex_fetch(const uint32_t *vals, uint32_t c, uint32_t end, bool vec, uint32_t lane,
                                         uint4 (&x)[EX_LOADS]) {
#pragma unroll
    for (uint32_t u = 0; u < EX_LOADS; ++u) {
        const uint32_t k = c + 128u * u + 4u * lane;
        if (vec && k + 4u <= end) {
            x[u] = ld_stream4(vals + k);
        } else {
            x[u].x = k < end ? ld_stream(vals + k) : 0u;
            x[u].y = k + 1u < end ? ld_stream(vals + k + 1u) : 0u;
            x[u].z = k + 2u < end ? ld_stream(vals + k + 2u) : 0u;
            x[u].w = k + 3u < end ? ld_stream(vals + k + 3u) : 0u;
        }
    }
}

// The window's pass mask: word k (values c + 32k .. c + 32k + 31) to lane k
// < 16, zero to lanes 16..31, and in fn the position of the first pass in
// words k+1 .. 15 (EX_NONE if none).  Lane l's four values of vector u are
// bits 4(l mod 8) .. +3 of word 4u + l/8; an OR over each group of eight
// lanes assembles the word, lane k fetches word k from its group, and a
// suffix minimum over the lanes gives fn.
template <class Test>
__device__ __forceinline__ uint32_t ex_bits(const uint4 (&x)[EX_LOADS], uint32_t lane, const Test &test,
                                            uint32_t &fn) {
    uint32_t wu[EX_LOADS];
#pragma unroll
    for (uint32_t u = 0; u < EX_LOADS; ++u) {
        uint32_t q = (uint32_t)test(x[u].x) | (uint32_t)test(x[u].y) << 1 | (uint32_t)test(x[u].z) << 2 |
                     (uint32_t)test(x[u].w) << 3;
        q <<= 4u * (lane & 7u);
        q |= __shfl_xor_sync(FULL, q, 1);
        q |= __shfl_xor_sync(FULL, q, 2);
        q |= __shfl_xor_sync(FULL, q, 4);
        wu[u] = q;
    }
    uint32_t bm = 0;
#pragma unroll
    for (uint32_t u = 0; u < EX_LOADS; ++u) {
        const uint32_t t = __shfl_sync(FULL, wu[u], 8u * (lane & 3u));
        if ((lane >> 2) == u) bm = t;
    }
    uint32_t f = bm ? 32u * lane + (uint32_t)__ffs(bm) - 1u : EX_NONE;
#pragma unroll
    for (uint32_t o = 1; o < 16u; o <<= 1) f = min(f, __shfl_down_sync(FULL, f, o));
    fn = __shfl_down_sync(FULL, f, 1);   // lane 31 keeps its own EX_NONE
    return bm;
}

template <int WPL, class Test>
__device__ __forceinline__ void exist_words(const uint32_t *rp, const uint32_t *vals, const Test test, uint32_t n,
                                            uint32_t n_words, uint32_t wb, uint32_t lane, uint32_t (&v)[WPL]) {
#pragma unroll
    for (int s = 0; s < WPL; ++s) v[s] = 0u;
    const uint32_t w_end = min(wb + 32u * WPL, n_words);   // the warp's words [wb, w_end)
    if (wb >= w_end) return;
    const bool vec = (reinterpret_cast<uintptr_t>(vals) & 15u) == 0;
    const uint32_t end = ld_stream(rp + min(32u * w_end, n));   // the end of the warp's run
    uint32_t c = ld_stream(rp + 32u * wb) & ~127u;               // the window
    // the warp's row pointers go to L2 ahead of their loads (a hint that
    // holds no registers)
    if ((reinterpret_cast<uintptr_t>(rp) & 15u) == 0) prefetch_range(rp, 32u * wb, min(32u * w_end, n) + 1u, lane);
    uint4 x[EX_LOADS];
    ex_fetch(vals, c, end, vec, lane, x);
    uint32_t fn;
    uint32_t bm = ex_bits(x, lane, test, fn);
    ex_fetch(vals, c + EX_WIN, end, vec, lane, x);               // the next window, in flight
    // row batches alternate between two registers, so a pending load is never copied
    ExRows ra, rb;
    ex_rows(ra, rp, wb, w_end, n, lane);
    ex_rows(rb, rp, wb + 4u, w_end, n, lane);
    auto batch = [&](uint32_t w0, const ExRows &rows) {
#pragma unroll 1
        for (uint32_t j = 0; j < 4u && w0 + j < w_end; ++j) {   // warp-uniform
            // this lane's row [lo, hi): lane 31's end is the next word's first row pointer
            const uint32_t lo = j == 0u ? rows.r[0] : j == 1u ? rows.r[1] : j == 2u ? rows.r[2] : rows.r[3];
            const uint32_t ln = j == 0u ? rows.r[1] : j == 1u ? rows.r[2] : j == 2u ? rows.r[3] : rows.tail;
            const uint32_t dn = __shfl_down_sync(FULL, lo, 1), up = __shfl_sync(FULL, ln, 0);
            const uint32_t hi = lane == 31u ? up : dn;
            bool hit = false;
            for (;;) {
                const int rl = (int)(lo - c), rh = (int)(hi - c);   // the row relative to the window
                const int a = max(rl, 0), b = min(rh, (int)EX_WIN);
                const uint32_t wa = (uint32_t)a >> 5;
                const uint32_t ma = __shfl_sync(FULL, bm, wa), fa = __shfl_sync(FULL, fn, wa);
                const uint32_t m = ma & (FULL << (a & 31));
                const int first = m ? (int)(32u * wa + (uint32_t)__ffs(m) - 1u) : (int)fa;   // first pass >= a
                hit = hit || (a < b && first < b);
                // the first value, past the window, of a row that has not passed yet
                const bool more = !hit && rh > (int)EX_WIN && rl < rh;
                const uint32_t nxt = __reduce_min_sync(FULL, more ? (uint32_t)max(rl, (int)EX_WIN) : 0xFFFFFFFFu);
                if (nxt == 0xFFFFFFFFu) break;
                const uint32_t cn = c + (nxt & ~127u);
                if (cn != c + EX_WIN) ex_fetch(vals, cn, end, vec, lane, x);   // a jump: not the window in flight
                c = cn;
                bm = ex_bits(x, lane, test, fn);
                ex_fetch(vals, c + EX_WIN, end, vec, lane, x);
            }
            const uint32_t word = __ballot_sync(FULL, hit), k = w0 + j - wb;
#pragma unroll
            for (int s = 0; s < WPL; ++s)
                if (lane == k / WPL && k % WPL == (uint32_t)s) v[s] = word;
        }
    };
    for (uint32_t w0 = wb; w0 < w_end; w0 += 8u) {
        batch(w0, ra);
        ex_rows(ra, rp, w0 + 8u, w_end, n, lane);
        if (w0 + 4u >= w_end) break;
        batch(w0 + 4u, rb);
        ex_rows(rb, rp, w0 + 12u, w_end, n, lane);
    }
}

// exist_words with the test's kind resolved at compile time (one dispatch per
// restriction, warp-uniform).
template <int WPL>
__device__ __forceinline__ void exist_words(const uint32_t *rp, const uint32_t *vals, const ValueTest &test,
                                            uint32_t n, uint32_t n_words, uint32_t wb, uint32_t lane,
                                            uint32_t (&v)[WPL]) {
    if (test.mode == ValueTest::FLOAT_CMP) {
        const float t = __uint_as_float(test.arg);
        if (test.cmp == HEDL_OP_DGE)
            exist_words<WPL>(rp, vals, FloatTest<HEDL_OP_DGE>{t}, n, n_words, wb, lane, v);
        else if (test.cmp == HEDL_OP_DLE)
            exist_words<WPL>(rp, vals, FloatTest<HEDL_OP_DLE>{t}, n, n_words, wb, lane, v);
        else
            exist_words<WPL>(rp, vals, FloatTest<HEDL_OP_DEQ>{t}, n, n_words, wb, lane, v);
    } else if (test.mode == ValueTest::ID_EQ)
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
