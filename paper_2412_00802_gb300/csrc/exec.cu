// Batched evaluation: one persistent interpreter kernel over a work queue of
// (task, tile) items (see plan.cpp for how a batch becomes tasks).
//
// Each CTA pops an item, waits (bounded) until every task it reads is
// complete, then its warps run the task over the tile.  A segment task is a
// stack machine whose values are bitset words (one register set per lane,
// deeper stack entries in shared memory), whose leaves load concept rows /
// slots, evaluate data ranges by ballot, or evaluate a lone role restriction
// by the warp's edge-stream CSR walk (role_stream).  A segment's result is
// written to its slot, or, for a hypothesis root, reduced against the example
// sets by popcount (the paper's coverage count, Algorithm 15) with one atomic
// per warp.  A role group (up to 64 restrictions sharing a role, direction
// and role depth) runs as two tasks: a transpose of its fillers into one or
// two 32-bit words per individual, and one bit-sliced walk that evaluates all
// of them.
//
// Waits never spin unbounded: each gives up after the plan's timeout, sets an
// abort flag and an error bit, and every CTA then leaves the kernel.
#include <cuda_runtime.h>

#include <cstddef>

#include "device_common.cuh"

namespace hedl {

namespace {

struct ExecArgs {
    KBView kb;
    uint8_t *ws;
    uint32_t *counts;     // [H][4] or null
    uint32_t *out_bits;   // [H][wp] or null
    uint32_t item_begin, item_end;
    uint32_t use_queue;   // 1: dynamic queue with dependency waits; 0: static striding, no waits
};

template <int NW, int WPL>
struct Smem {
    uint32_t stk[NW][STACK_MAX][WPL][32];
    uint64_t leaf[NW][PF_SLOTS];   // per warp: the segment's first leaf rows (bit 0 set: a slot)
    uint32_t item;
    uint32_t ok;
    uint32_t pad[2];
    uint32_t filler[1];   // staged plans: the segment's filler row (wp words) from here on
};

// The last group with item_begin <= item.  A CTA's items only grow (the queue
// hands them out in order; static striding steps forward), so the search
// starts at the CTA's previous group: a few steps forward, else a binary
// search over the groups after it.
__device__ __forceinline__ uint32_t find_group(const Group *groups, uint32_t n_groups, uint32_t item, uint32_t from) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (from + 1 >= n_groups || groups[from + 1].item_begin > item) return from;
        ++from;
    }
    uint32_t lo = from, hi = n_groups;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (groups[mid].item_begin <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <int NW, int WPL, bool STAGE, int BLK, bool CONCRETE>
__device__ void run_tile(const ExecArgs &A, const PlanHeader &hd, const Seg &seg, uint32_t tile,
                         Smem<NW, WPL> &sm, uint32_t *slots, uint32_t *acc) {
    const KBView &kb = A.kb;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const DInsn *code = reinterpret_cast<const DInsn *>(A.ws + hd.off_code) + seg.code_off;
    // a warp covers ww * WPL words a round; with ww < 32, lanes ww..31 hold
    // words of no one: every load, store and walk stops at the warp's limit
    const uint32_t ww = hd.warp_words;
    const uint32_t rounds = hd.tile_words / (NW * ww * WPL);
    // The segment's first PF concept-row and slot leaves, in code order: each
    // round loads them all at once (their latencies overlap), and the stack
    // machine takes the k-th such leaf from pf[k] instead of loading it where
    // it stands.  The warp builds the table with one ballot per 32
    // instructions.
    constexpr int PF = WPL == 1 ? PF_SLOTS : 2;
    uint32_t n_pf = 0;
    for (uint32_t b0 = 0; b0 < seg.code_len && n_pf < (uint32_t)PF; b0 += 32) {
        const uint32_t pc = b0 + lane;
        uint64_t addr = 0;
        bool leaf = false;
        if (pc < seg.code_len) {
            const DInsn d = code[pc];
            const uint32_t op = d.op & 0xFFu;
            if (op == D_ATOM) {
                leaf = true;
                addr = reinterpret_cast<uint64_t>(kb.concepts + (uint64_t)d.a * kb.wp);
            } else if (op == D_SLOT) {
                leaf = true;
                addr = reinterpret_cast<uint64_t>(slots + (uint64_t)d.ref * kb.wp) | 1ull;
            }
        }
        const uint32_t m = __ballot_sync(FULL, leaf);
        const uint32_t rank = n_pf + __popc(m & ((1u << lane) - 1u));
        if (leaf && rank < (uint32_t)PF) sm.leaf[warp][rank] = addr;
        n_pf = min((uint32_t)PF, n_pf + (uint32_t)__popc(m));
    }
    __syncwarp();
    const bool score = seg.hyp != NO_HYP && A.counts;
    uint32_t tp = 0, fp = 0;
    // the leaf rows (and example rows) of one round, loaded together
    auto prefetch = [&](uint32_t wb, uint32_t (&pf)[PF][WPL], uint32_t (&pv)[WPL], uint32_t (&nv)[WPL]) {
        const uint32_t lim_p = min(kb.wp, wb + ww * WPL);   // padded row words
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            if ((uint32_t)k < n_pf) {
                const uint64_t a = sm.leaf[warp][k];
                if (a & 1ull) load_row_rw<WPL>(reinterpret_cast<const uint32_t *>(a & ~1ull), wb, lane, lim_p, pf[k]);
                else load_row_ro<WPL>(reinterpret_cast<const uint32_t *>(a), wb, lane, lim_p, pf[k]);
            } else {
#pragma unroll
                for (int s = 0; s < WPL; ++s) pf[k][s] = 0u;
            }
        }
        if (score) {
            load_row_ro<WPL>(kb.pos, wb, lane, lim_p, pv);
            load_row_ro<WPL>(kb.neg, wb, lane, lim_p, nv);
        } else {
#pragma unroll
            for (int s = 0; s < WPL; ++s) pv[s] = nv[s] = 0u;
        }
    };
    // the stack machine over one round's words
    auto evaluate = [&](uint32_t wb, const uint32_t (&pf)[PF][WPL], const uint32_t (&pv)[WPL],
                        const uint32_t (&nv)[WPL]) {
        const uint32_t lim_p = min(kb.wp, wb + ww * WPL);   // padded row words
        const uint32_t lim_w = min(kb.w, wb + ww * WPL);    // words holding individuals
        uint32_t n_used = 0;   // concept-row and slot leaves met so far this round
        uint32_t top[WPL];
        uint32_t sp = 0;  // values on the stack, top included
        for (uint32_t pc = 0; pc < seg.code_len; ++pc) {
            const DInsn d = code[pc];
            const uint32_t op = d.op & 0xFFu;
            if (op == D_NOT) {
#pragma unroll
                for (int s = 0; s < WPL; ++s)
                    top[s] = ~top[s] & tail_mask(wb + lane * WPL + s, kb.w, kb.n);
                continue;
            }
            if (op == D_AND || op == D_OR) {
                sp -= 1;
#pragma unroll
                for (int s = 0; s < WPL; ++s) {
                    uint32_t o = sm.stk[warp][sp - 1][s][lane];
                    top[s] = op == D_AND ? (top[s] & o) : (top[s] | o);
                }
                continue;
            }
            // a leaf: spill the current top, compute the new one
            if (sp > 0) {
#pragma unroll
                for (int s = 0; s < WPL; ++s) sm.stk[warp][sp - 1][s][lane] = top[s];
            }
            sp += 1;
            switch (op) {
            case D_ATOM:
            case D_SLOT:
                if (n_used < n_pf) {   // loaded at the start of the round
#pragma unroll
                    for (int s = 0; s < WPL; ++s) {
                        uint32_t x = pf[0][s];
#pragma unroll
                        for (int k = 1; k < PF; ++k)
                            if ((uint32_t)k == n_used) x = pf[k][s];
                        top[s] = x;
                    }
                } else if (op == D_ATOM) {
                    load_row_ro<WPL>(kb.concepts + (uint64_t)d.a * kb.wp, wb, lane, lim_p, top);
                } else {
                    load_row_rw<WPL>(slots + (uint64_t)d.ref * kb.wp, wb, lane, lim_p, top);
                }
                ++n_used;
                break;
            case D_TOP:
#pragma unroll
                for (int s = 0; s < WPL; ++s) top[s] = tail_mask(wb + lane * WPL + s, kb.w, kb.n);
                break;
            case D_BOT:
#pragma unroll
                for (int s = 0; s < WPL; ++s) top[s] = 0u;
                break;
            case D_DATA:
                if ((d.op >> 8) & 3u) {   // a numeric (bit 8) or string (bit 9) concrete role
                    if constexpr (CONCRETE) {
                        const bool str = (d.op >> 9) & 1u;
                        const uint32_t *rp = str ? kb.str[d.a].rp : kb.num[d.a].rp;
                        const uint32_t *vals =
                            str ? kb.str[d.a].ids : reinterpret_cast<const uint32_t *>(kb.num[d.a].vals);
                        exist_words<WPL>(rp, vals, value_test(kb, d.op, d.b), kb.n, lim_w, wb, lane, top);
                    }
                } else
                    data_words<WPL>(kb.props + (uint64_t)d.a * kb.prop_stride, (d.op >> 16) & 0xFFu,
                                    __uint_as_float(d.b), kb.n, lim_w, wb, lane, top);
                break;
            default: {  // D_ROLE
                const uint32_t inv = (d.op >> 8) & 1u;
                const DevCSR g = kb.csr[2u * d.a + inv];
                if constexpr (STAGE) {
                    const uint32_t kind = (d.op >> 16) & 0xFFu;
                    role_stream<WPL, BLK>(g, sm.filler, kind, d.b, kb.n, lim_w, wb, lane, top, kind == HEDL_OP_FORALL);
                } else {
                    const uint32_t *filler = (d.ref & REF_SLOT) ? slots + (uint64_t)(d.ref & ~REF_SLOT) * kb.wp
                                                                : kb.concepts + (uint64_t)d.ref * kb.wp;
                    role_stream<WPL, BLK>(g, filler, (d.op >> 16) & 0xFFu, d.b, kb.n, lim_w, wb, lane, top);
                }
                break;
            }
            }
        }
        if (seg.out_slot != NO_SLOT) store_row<WPL>(slots + (uint64_t)seg.out_slot * kb.wp, wb, lane, lim_p, top);
        if (seg.hyp != NO_HYP) {
            if (A.out_bits) store_row<WPL>(A.out_bits + (uint64_t)seg.hyp * kb.wp, wb, lane, lim_p, top);
            if (score) {
#pragma unroll
                for (int s = 0; s < WPL; ++s) {
                    tp += __popc(top[s] & pv[s]);
                    fp += __popc(top[s] & nv[s]);
                }
            }
        }
    };
    // one round at a time: the round's leaf rows are all requested before the
    // first instruction runs (requesting the next round's as well was slower:
    // twice the prefetch registers, more spills)
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t wb = tile * hd.tile_words + (r * NW + warp) * ww * WPL;
        if (wb >= kb.wp) break;
        uint32_t pf[PF][WPL], pv[WPL], nv[WPL];
        prefetch(wb, pf, pv, nv);
        evaluate(wb, pf, pv, nv);
    }
    if (seg.hyp != NO_HYP && A.counts) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tp += __shfl_xor_sync(FULL, tp, o);
            fp += __shfl_xor_sync(FULL, fp, o);
        }
        if (lane == 0) {
            if (tp) atomicAdd(acc + 2u * seg.hyp, tp);
            if (fp) atomicAdd(acc + 2u * seg.hyp + 1u, fp);
        }
    }
}

// ------------------------------------------------------------------ bit-sliced role groups
// 32 x 32 bit transpose across a warp: lane r holds row r (bit c = column c)
// on entry and column r on exit.  Five butterfly stages swap the
// off-diagonal blocks of size 16, 8, 4, 2, 1.
__device__ __forceinline__ uint32_t transpose32(uint32_t x, uint32_t lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const uint32_t j = 16u >> st, m = masks[st];
        const uint32_t t = __shfl_xor_sync(FULL, x, j);
        x = (lane & j) ? ((x & ~m) | ((t >> j) & m)) : ((x & m) | ((t & m) << j));
    }
    return x;
}

// Transpose task: word p of FT[i], bit s = slice 32p + s's filler at
// individual i (its complement for REF_NEG slices), one 32-word pass per warp
// at a time; lane s reads slice 32p + s's row.
template <int NW, int P>
__device__ void run_transpose(const ExecArgs &A, const PlanHeader &hd, const RGroup *gp, uint32_t tile,
                              const uint32_t *slots) {
    const KBView &kb = A.kb;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t n = gp->n;
    const uint32_t *src[P];
    uint32_t x[P];
    bool on[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const uint32_t s = 32u * q + lane;
        on[q] = s < n;
        const uint32_t ref = on[q] ? gp->filler[s] : 0u;
        const uint32_t id = ref & REF_ID;
        src[q] = (ref & REF_SLOT) ? slots + (uint64_t)id * kb.wp : kb.concepts + (uint64_t)id * kb.wp;
        x[q] = (ref & REF_NEG) ? FULL : 0u;
    }
    uint32_t *ft = reinterpret_cast<uint32_t *>(A.ws + gp->ft_off);
    const uint32_t passes = hd.tile_words / (NW * 32u);
    for (uint32_t p = 0; p < passes; ++p) {
        const uint32_t wb = tile * hd.tile_words + (p * NW + warp) * 32u;
        if (wb >= kb.w) break;
        for (uint32_t j = 0; j < 32u; ++j) {
            const uint32_t w = wb + j;
            if (w >= kb.w) break;
            uint32_t t[P];
#pragma unroll
            for (int q = 0; q < P; ++q) t[q] = transpose32(on[q] ? (src[q][w] ^ x[q]) : 0u, lane);
            if constexpr (P == 1) ft[32ull * w + lane] = t[0];
            else reinterpret_cast<uint2 *>(ft)[32ull * w + lane] = make_uint2(t[0], t[1]);
        }
    }
}

// v = v + x per slice, saturating at 7 (planes c0 < c1 < c2).
__device__ __forceinline__ void sat_add1(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t x) {
    x &= ~(c0 & c1 & c2);
    const uint32_t k1 = c0 & x;
    c0 ^= x;
    const uint32_t k2 = c1 & k1;
    c1 ^= k1;
    c2 |= k2;
}

// a = a + b per slice (3-bit values), saturating at 7.
__device__ __forceinline__ void sat_add3(uint32_t &a0, uint32_t &a1, uint32_t &a2, uint32_t b0, uint32_t b1,
                                         uint32_t b2) {
    const uint32_t s0 = a0 ^ b0, k0 = a0 & b0;
    const uint32_t s1 = a1 ^ b1 ^ k0, k1 = (a1 & b1) | (k0 & (a1 ^ b1));
    const uint32_t s2 = a2 ^ b2 ^ k1, k2 = (a2 & b2) | (k1 & (a2 ^ b2));
    a0 = s0 | k2;
    a1 = s1 | k2;
    a2 = s2 | k2;
}

constexpr uint32_t HEAVY_ROW = 64;   // longer rows are walked by the whole warp
constexpr uint32_t WALK_BUF = 256;   // 32-bit words of a warp's window buffer

// Walk task: for each individual, the saturating per-slice count of its
// successors' FT words (P words each: 32 P slices), mapped through the
// group's truth tables, transposed back into the output slots (4 / P words
// per lane per store).  The warp takes its words 4 / P at a time (their
// individuals' rows form one contiguous edge range) and streams that range in
// windows of WALK_BUF / P edges: lane e loads edges e, e + 32, ...
// of the window (coalesced), gathers their FT words and puts them in a
// per-warp shared-memory buffer; then each lane adds the buffer entries of its
// own rows.  The next window's edges are loaded while the current window's FT
// words are gathered, and windows that hold no light row's edge are skipped.
// Rows longer than HEAVY_ROW are walked by the whole warp, 32 edges at a time,
// and their counts reduced across lanes.
template <int NW, int P>
__device__ void run_walk(const ExecArgs &A, const PlanHeader &hd, const RGroup *gp, uint32_t tile,
                         uint32_t *slots, uint32_t *buf) {
    constexpr uint32_t LOADS = WALK_BUF / (32u * P);   // edges a lane gathers per window
    constexpr uint32_t WIN = 32u * LOADS;
    constexpr uint32_t CW = 4u / P;                    // words per chunk: 4 x 3 x P counters a lane
    const KBView &kb = A.kb;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const DevCSR g = kb.csr[gp->role2];
    const uint32_t *__restrict__ rp = g.rp;
    const uint32_t *__restrict__ col = g.col;
    const uint32_t *ft = reinterpret_cast<const uint32_t *>(A.ws + gp->ft_off);
    const uint32_t n = gp->n;
    // one FT entry (P words) of individual b
    auto ft_at = [&](uint32_t b, uint32_t (&o)[P]) {
        if constexpr (P == 1) {
            o[0] = ft[b];
        } else {
            const uint2 q = reinterpret_cast<const uint2 *>(ft)[b];
            o[0] = q.x;
            o[1] = q.y;
        }
    };
    const uint32_t passes = hd.tile_words / (NW * 32u);
    for (uint32_t p = 0; p < passes; ++p) {
        const uint32_t wb = tile * hd.tile_words + (p * NW + warp) * 32u;
        if (wb >= kb.wp) break;
        for (uint32_t jj = 0; jj < 32u; jj += CW) {
            if (wb + jj >= kb.wp) break;   // wp and wb are multiples of 4: whole chunks
            uint32_t lo[CW], hi[CW];
            bool light[CW], heavy[CW];
#pragma unroll
            for (uint32_t q = 0; q < CW; ++q) {
                const uint32_t w = wb + jj + q, i = w * 32u + lane;
                lo[q] = hi[q] = 0;
                if (w < kb.w && i < kb.n) {
                    lo[q] = ld_stream(rp + i);
                    hi[q] = ld_stream(rp + i + 1);
                }
                heavy[q] = hi[q] - lo[q] > HEAVY_ROW;
                light[q] = !heavy[q] && hi[q] > lo[q];
            }
            // the chunk's edge range ends at its last individual's row end
            uint32_t hmax = hi[0];
#pragma unroll
            for (uint32_t q = 1; q < CW; ++q) hmax = max(hmax, hi[q]);
            const uint32_t E1 = __reduce_max_sync(FULL, hmax);
            // first edge at or after `at` that some light row of the chunk holds (E1 if none)
            auto next_light = [&](uint32_t at) {
                uint32_t m = E1;
#pragma unroll
                for (uint32_t q = 0; q < CW; ++q)
                    if (light[q] && hi[q] > at) m = min(m, max(lo[q], at));
                return __reduce_min_sync(FULL, m);
            };
            uint32_t c0[CW][P], c1[CW][P], c2[CW][P];
#pragma unroll
            for (uint32_t q = 0; q < CW; ++q)
#pragma unroll
                for (int k = 0; k < P; ++k) c0[q][k] = c1[q][k] = c2[q][k] = 0;
            uint32_t base = next_light(0);
            uint32_t cn[LOADS];
            auto fetch = [&](uint32_t at) {
#pragma unroll
                for (uint32_t u = 0; u < LOADS; ++u) {
                    const uint32_t e = at + 32u * u + lane;
                    cn[u] = e < E1 ? ld_stream(col + e) : 0u;
                }
            };
            if (base < E1) fetch(base);
            while (base < E1) {   // warp-uniform
                uint32_t b[LOADS];
#pragma unroll
                for (uint32_t u = 0; u < LOADS; ++u) b[u] = cn[u];
                const uint32_t nb = base + WIN, next = next_light(nb);
                if (next < E1) fetch(next);
                uint32_t x[LOADS][P];
#pragma unroll
                for (uint32_t u = 0; u < LOADS; ++u) {
                    if (base + 32u * u + lane < E1) {
                        ft_at(b[u], x[u]);
                    } else {
#pragma unroll
                        for (int k = 0; k < P; ++k) x[u][k] = 0u;
                    }
                }
#pragma unroll
                for (uint32_t u = 0; u < LOADS; ++u) {   // one P-word store per lane: no bank conflicts
                    if constexpr (P == 1) buf[32u * u + lane] = x[u][0];
                    else reinterpret_cast<uint2 *>(buf)[32u * u + lane] = make_uint2(x[u][0], x[u][1]);
                }
                __syncwarp();
#pragma unroll
                for (uint32_t q = 0; q < CW; ++q) {
                    if (!light[q]) continue;
                    const uint32_t k1 = min(hi[q], nb);
                    for (uint32_t e = max(lo[q], base); e < k1; ++e) {
                        if constexpr (P == 1) {
                            sat_add1(c0[q][0], c1[q][0], c2[q][0], buf[e - base]);
                        } else {
                            const uint2 y = reinterpret_cast<const uint2 *>(buf)[e - base];
                            sat_add1(c0[q][0], c1[q][0], c2[q][0], y.x);
                            sat_add1(c0[q][1], c1[q][1], c2[q][1], y.y);
                        }
                    }
                }
                __syncwarp();
                base = next;
            }
            uint32_t outw[P][CW];
#pragma unroll
            for (uint32_t q = 0; q < CW; ++q) {
                uint32_t hm = __ballot_sync(FULL, heavy[q]);
                while (hm) {
                    const uint32_t h = __ffs(hm) - 1;
                    hm &= hm - 1;
                    const uint32_t hlo = __shfl_sync(FULL, lo[q], h), hhi = __shfl_sync(FULL, hi[q], h);
                    uint32_t d0[P], d1[P], d2[P];
#pragma unroll
                    for (int k = 0; k < P; ++k) d0[k] = d1[k] = d2[k] = 0;
                    for (uint32_t e = hlo + lane; e < hhi; e += 32u) {
                        uint32_t y[P];
                        ft_at(ld_stream(col + e), y);
#pragma unroll
                        for (int k = 0; k < P; ++k) sat_add1(d0[k], d1[k], d2[k], y[k]);
                    }
#pragma unroll
                    for (int k = 0; k < P; ++k) {
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const uint32_t e0 = __shfl_xor_sync(FULL, d0[k], o), e1 = __shfl_xor_sync(FULL, d1[k], o);
                            const uint32_t e2 = __shfl_xor_sync(FULL, d2[k], o);
                            sat_add3(d0[k], d1[k], d2[k], e0, e1, e2);
                        }
                        if (lane == h) {
                            c0[q][k] = d0[k];
                            c1[q][k] = d1[k];
                            c2[q][k] = d2[k];
                        }
                    }
                }
                const uint32_t w = wb + jj + q;
                const bool valid = w < kb.w && w * 32u + lane < kb.n;
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    uint32_t r = 0;
#pragma unroll
                    for (int v = 0; v < 8; ++v) {
                        const uint32_t m = ((v & 4) ? c2[q][k] : ~c2[q][k]) & ((v & 2) ? c1[q][k] : ~c1[q][k]) &
                                           ((v & 1) ? c0[q][k] : ~c0[q][k]);
                        r |= m & gp->want[k][v];   // the group's truth table (cached, read per word)
                    }
                    r = valid ? r : 0u;
                    outw[k][q] = transpose32(r, lane);   // lane s: slice 32k + s's word w
                }
            }
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const uint32_t s = 32u * k + lane;
                if (s < n) {   // aligned: wb + jj is a multiple of CW
                    uint32_t *dst = slots + (uint64_t)gp->out[s] * kb.wp + wb + jj;
                    if constexpr (CW == 4)
                        *reinterpret_cast<uint4 *>(dst) = make_uint4(outw[k][0], outw[k][1], outw[k][2], outw[k][3]);
                    else
                        *reinterpret_cast<uint2 *>(dst) = make_uint2(outw[k][0], outw[k][1]);
                }
            }
        }
    }
}

// Bounded wait for every producer segment of `seg` (thread 0 only).
__device__ bool wait_deps(const PlanHeader &hd, const uint32_t *deps, const Seg &seg, uint32_t *done,
                          Counters *ctr) {
    for (uint32_t k = 0; k < seg.dep_cnt; ++k) {
        const uint32_t *flag = done + deps[seg.dep_off + k];
        if (ld_acquire(flag) >= hd.n_tiles) continue;
        const uint64_t t0 = global_ns();
        uint64_t spins = 0;
        const uint64_t max_spins = hd.timeout_ns / 16 + 1000000ull;
        while (ld_acquire(flag) < hd.n_tiles) {
            if (*(volatile uint32_t *)&ctr->abort) return false;
            if (global_ns() - t0 > hd.timeout_ns || ++spins > max_spins) {
                atomicOr(&ctr->err, ST_TIMEOUT);
                atomicExch(&ctr->abort, 1u);
                return false;
            }
            __nanosleep(128);
        }
    }
    return true;
}

// Copy the segment's filler row into shared memory (all threads of the CTA).
// A FORALL filler is staged complemented (REF_NEG), so the walk counts
// successors outside C without a per-edge complement.
__device__ __forceinline__ void stage_filler(const KBView &kb, const uint32_t *slots, uint32_t ref, uint32_t *dst) {
    const uint32_t id = ref & REF_ID;
    const uint32_t *src = (ref & REF_SLOT) ? slots + (uint64_t)id * kb.wp : kb.concepts + (uint64_t)id * kb.wp;
    const uint32_t x = (ref & REF_NEG) ? 0xFFFFFFFFu : 0u;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (uint32_t q = threadIdx.x; q < kb.wp / 4; q += blockDim.x) {
        uint4 v = s4[q];
        d4[q] = make_uint4(v.x ^ x, v.y ^ x, v.z ^ x, v.w ^ x);
    }
}

// Register budget: every shape is compiled for 768 resident threads per SM
// (80 registers a thread; the prefetching stack machine and the windowed walks
// spill heavily at 64); FULL ones for 2,048 (32 registers, full occupancy, at
// the price of spills).  GROUPS = false leaves the role groups' transposes and
// walks out (for plans without role groups: a lone hypothesis, concrete-role
// restrictions); the rest fits 64 registers, so that build keeps 1,024
// threads per SM for the latency-bound lone walks and value streams.
// CONCRETE = false leaves the concrete-role value walk out, for KBs that have
// no concrete roles: its registers would otherwise raise the spills of the
// whole stack machine.
template <int NW, int WPL, bool STAGE, int BLK, bool FULL = false, bool GROUPS = true, bool CONCRETE = true>
__global__ void __launch_bounds__(NW * 32, (FULL ? 64 : (GROUPS ? 24 : 32)) / NW) exec_kernel(ExecArgs A) {
    // the host sizes the dynamic shared memory as stack_smem_bytes + 16 (+ a staged filler)
    using SmemT = Smem<NW, WPL>;
    static_assert(offsetof(SmemT, filler) ==
                      sizeof(uint32_t) * NW * STACK_MAX * WPL * 32 + sizeof(uint64_t) * NW * PF_SLOTS + 16,
                  "the shared-memory layout and its host-side size disagree");
    extern __shared__ __align__(16) uint8_t smem_raw[];
    Smem<NW, WPL> &sm = *reinterpret_cast<Smem<NW, WPL> *>(smem_raw);
    const PlanHeader hd = *reinterpret_cast<const PlanHeader *>(A.ws);
    const Seg *segs = reinterpret_cast<const Seg *>(A.ws + hd.off_segs);
    const Group *groups = reinterpret_cast<const Group *>(A.ws + hd.off_groups);
    const uint32_t *gsegs = reinterpret_cast<const uint32_t *>(A.ws + hd.off_gsegs);
    const uint32_t *deps = reinterpret_cast<const uint32_t *>(A.ws + hd.off_deps);
    Counters *ctr = reinterpret_cast<Counters *>(A.ws + hd.off_ctr);
    uint32_t *done = reinterpret_cast<uint32_t *>(ctr + 1);
    uint32_t *acc = done + hd.n_segs + 1;
    uint32_t *slots = reinterpret_cast<uint32_t *>(A.ws + hd.off_slots);
    const RGroup *rgroups = reinterpret_cast<const RGroup *>(A.ws + hd.off_rgroups);

    // Thread 0 claims the next item as soon as the current one may start (its
    // dependencies are done), so the claim's round trip overlaps the work.
    // Items are claimed in queue order and a CTA holds at most two, the one it
    // runs and the next; every dependency points to an earlier item, so the
    // earliest unfinished item is always running and the queue drains.
    uint32_t stride_next = A.item_begin + blockIdx.x;
    uint32_t nxt = A.item_end;   // thread 0: the item claimed while the current one runs
    uint32_t g = 0;              // the current item's group
    if (threadIdx.x == 0) sm.item = A.use_queue ? A.item_begin + atomicAdd(&ctr->head, 1u) : stride_next;
    for (;;) {
        __syncthreads();
        const uint32_t item = sm.item;
        stride_next += gridDim.x;
        if (item >= A.item_end) break;
        g = find_group(groups, hd.n_groups, item, g);
        const Group grp = groups[g];
        const uint32_t local = item - grp.item_begin;
        const uint32_t tile = local / grp.n_segs;
        const uint32_t sidx = gsegs[grp.seg_begin + local % grp.n_segs];
        const Seg seg = segs[sidx];
        if (A.use_queue) {
            if (threadIdx.x == 0) {
                const bool ok = wait_deps(hd, deps, seg, done, ctr);
                sm.ok = ok ? 1u : 0u;
                if (ok) nxt = A.item_begin + atomicAdd(&ctr->head, 1u);
            }
            __syncthreads();
            if (!sm.ok) break;
        }
        if (seg.kind != TASK_SEGMENT && !GROUPS) {
            // a build without role groups was given a plan with them (the host never does this)
            if (threadIdx.x == 0) {
                atomicOr(&ctr->err, ST_DEVICE_CHECK);
                atomicExch(&ctr->abort, 1u);
            }
        } else if (seg.kind == TASK_TRANSPOSE) {
            if constexpr (GROUPS) {
                const RGroup *gp = rgroups + seg.code_off;
                if (gp->parts == 1) run_transpose<NW, 1>(A, hd, gp, tile, slots);
                else run_transpose<NW, MAX_PARTS>(A, hd, gp, tile, slots);
            }
        } else if (seg.kind == TASK_WALK) {
            if constexpr (GROUPS) {
                // the warp's stack (unused by a walk) holds its window of gathered FT words
                const RGroup *gp = rgroups + seg.code_off;
                uint32_t *buf = &sm.stk[threadIdx.x >> 5][0][0][0];
                if (gp->parts == 1) run_walk<NW, 1>(A, hd, gp, tile, slots, buf);
                else run_walk<NW, MAX_PARTS>(A, hd, gp, tile, slots, buf);
            }
        } else {
            if constexpr (STAGE) {
                if (seg.filler != NO_FILLER) {
                    stage_filler(A.kb, slots, seg.filler, sm.filler);
                    __syncthreads();
                }
            }
            run_tile<NW, WPL, STAGE, BLK, CONCRETE>(A, hd, seg, tile, sm, slots, acc);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (A.use_queue) {
                __threadfence();
                atomicAdd(done + sidx, 1u);
                sm.item = *(volatile uint32_t *)&ctr->abort ? A.item_end : nxt;
            } else {
                sm.item = stride_next;
            }
        }
    }
}

// (TP, FP) accumulators -> (TP, FP, FN, TN); records a device error on the handle.
__global__ void finalize_kernel(KBView kb, const uint8_t *ws, uint32_t *counts) {
    const PlanHeader *hd = reinterpret_cast<const PlanHeader *>(ws);
    const Counters *ctr = reinterpret_cast<const Counters *>(ws + hd->off_ctr);
    const uint32_t *acc = reinterpret_cast<const uint32_t *>(ctr + 1) + hd->n_segs + 1;
    if (blockIdx.x == 0 && threadIdx.x == 0 && ctr->err) atomicOr(kb.status, ctr->err);
    if (!counts) return;
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < hd->n_hyps; h += gridDim.x * blockDim.x) {
        const uint32_t tp = acc[2 * h], fp = acc[2 * h + 1];
        uint4 c = make_uint4(tp, fp, kb.n_pos - tp, kb.n_neg - fp);
        *reinterpret_cast<uint4 *>(counts + 4ull * h) = c;
    }
}

using KernelFn = void (*)(ExecArgs);

// Instantiated launch shapes: warps x words per lane x staging x chunks per block
// (1- and 2-warp CTAs only with one word per lane and no staging).
template <bool STAGE, int BLK>
KernelFn pick_t(uint32_t warps, uint32_t wpl) {
    if (wpl == 4) {
        if (warps == 4) return exec_kernel<4, 4, STAGE, BLK>;
        if (warps == 16) return exec_kernel<16, 4, STAGE, BLK>;
        return exec_kernel<8, 4, STAGE, BLK>;
    }
    if constexpr (!STAGE) {
        if (warps == 1) return exec_kernel<1, 1, false, BLK>;
        if (warps == 2) return exec_kernel<2, 1, false, BLK>;
    }
    if (warps == 4) return exec_kernel<4, 1, STAGE, BLK>;
    if (warps == 16) return exec_kernel<16, 1, STAGE, BLK>;
    if (warps == 32) return exec_kernel<32, 1, STAGE, BLK>;
    return exec_kernel<8, 1, STAGE, BLK>;
}

KernelFn pick(const Tuning &t, bool stage, bool groups, bool concrete) {
    if (!concrete && !t.full_occupancy && t.warps == 8 && t.wpl == 1 && !stage) {   // the common shapes
        if (!groups)
            return t.role_block == 4 ? exec_kernel<8, 1, false, 4, false, false, false>
                                     : exec_kernel<8, 1, false, 8, false, false, false>;
        return t.role_block == 4 ? exec_kernel<8, 1, false, 4, false, true, false>
                                 : exec_kernel<8, 1, false, 8, false, true, false>;
    }
    if (!groups && !t.full_occupancy && t.warps == 8 && t.wpl == 1 && !stage)   // no role groups: 64 registers
        return t.role_block == 4 ? exec_kernel<8, 1, false, 4, false, false> : exec_kernel<8, 1, false, 8, false, false>;
    if (t.full_occupancy && t.warps == 8 && t.wpl == 1 && !stage)
        return t.role_block == 4 ? exec_kernel<8, 1, false, 4, true> : exec_kernel<8, 1, false, 8, true>;
    if (t.role_block == 4) return stage ? pick_t<true, 4>(t.warps, t.wpl) : pick_t<false, 4>(t.warps, t.wpl);
    return stage ? pick_t<true, 8>(t.warps, t.wpl) : pick_t<false, 8>(t.warps, t.wpl);
}

size_t smem_bytes(const hedl_kb *kb, const Tuning &t, bool stage) {
    size_t b = stack_smem_bytes(t) + 16;   // stacks, leaf tables, then item / ok / pad
    if (stage) b += 4ull * kb->wp;
    return b;
}

}  // namespace

bool use_staging(const hedl_kb *kb, const Tuning &t) {
    return t.stage && t.warps >= 4 && smem_bytes(kb, t, true) <= kb->smem_optin;
}

size_t exec_smem_bytes(const Tuning &t) { return stack_smem_bytes(t) + 16; }

int exec_occupancy(const hedl_kb *kb, const Tuning &t, bool groups, int *blocks_per_sm) {
    const bool stage = use_staging(kb, t);
    KernelFn fn = pick(t, stage, groups, kb->has_concrete());
    size_t smem = smem_bytes(kb, t, stage);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, (int)(t.warps * 32), smem);
    return e;
}

int launch_exec(const hedl_kb *kb, const PlanImpl *p, uint32_t *counts, uint32_t *out_bits, void *ws,
                void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const Tuning &t = p->tuning;
    KernelFn fn = pick(t, p->staged, p->n_rgroups > 0, kb->has_concrete());
    size_t smem = smem_bytes(kb, t, p->staged);
    int bps = p->bps;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    if (t.ctas_per_sm && (int)t.ctas_per_sm < bps) bps = (int)t.ctas_per_sm;
    ExecArgs A{};
    A.kb = kb->view();
    A.ws = (uint8_t *)ws;
    A.counts = counts;
    A.out_bits = out_bits;
    const uint32_t n_items = p->info.n_items;
    if (p->flags & HEDL_LEVELS) {
        // one launch per level; items of a level are independent
        A.use_queue = 0;
        for (uint32_t l = 0; l < p->info.n_levels; ++l) {
            A.item_begin = p->level_items[l];
            A.item_end = p->level_items[l + 1];
            uint32_t n = A.item_end - A.item_begin;
            if (!n) continue;
            uint32_t grid = std::min<uint32_t>(n, (uint32_t)(bps * kb->n_sms));
            fn<<<grid, t.warps * 32, smem, s>>>(A);
            cudaError_t le = cudaGetLastError();
            if (le != cudaSuccess) return le;
        }
    } else {
        A.use_queue = 1;
        A.item_begin = 0;
        A.item_end = n_items;
        uint32_t grid = std::min<uint32_t>(std::max<uint32_t>(n_items, 1), (uint32_t)(bps * kb->n_sms));
        fn<<<grid, t.warps * 32, smem, s>>>(A);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return le;
    }
    finalize_kernel<<<std::max<uint32_t>(1, std::min<uint32_t>((p->n_hyps + 255) / 256, 1024)), 256, 0, s>>>(
        kb->view(), (const uint8_t *)ws, counts);
    return cudaGetLastError();
}

}  // namespace hedl
