// The plain path: one kernel launch per DL operation per hypothesis, each
// reading and writing full bitset rows, then one coverage-count launch per
// hypothesis.  This is the paper's own execution model (one GPU kernel per
// operator, Algorithms 2/4/6/8/10, then the coverage count of Algorithm 15),
// kept as the baseline that batching is measured against.  The operator
// kernels share the device building blocks of the batched interpreter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "device_common.cuh"

namespace hedl {

namespace {

constexpr int PT = 256;  // threads per block of the plain kernels

// Conjunction / disjunction / negation / constants over whole rows, four
// words (128 bits) per thread.
__global__ void bool_kernel(uint32_t op, const uint32_t *__restrict__ x, const uint32_t *__restrict__ y,
                            uint32_t *__restrict__ out, uint32_t wp, uint32_t n_words, uint32_t n) {
    const uint32_t quads = wp / 4;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < quads; q += gridDim.x * blockDim.x) {
        uint4 a = make_uint4(0, 0, 0, 0), b = make_uint4(0, 0, 0, 0);
        if (x) a = *reinterpret_cast<const uint4 *>(x + 4 * q);
        if (y) b = *reinterpret_cast<const uint4 *>(y + 4 * q);
        uint32_t r[4] = {a.x, a.y, a.z, a.w};
        const uint32_t o[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const uint32_t m = tail_mask(4 * q + s, n_words, n);
            if (op == HEDL_OP_AND) r[s] &= o[s];
            else if (op == HEDL_OP_OR) r[s] |= o[s];
            else if (op == HEDL_OP_NOT) r[s] = ~r[s] & m;
            else if (op == HEDL_OP_TOP) r[s] = m;
            else if (op == HEDL_OP_BOT) r[s] = 0u;
        }
        *reinterpret_cast<uint4 *>(out + 4 * q) = make_uint4(r[0], r[1], r[2], r[3]);
    }
}

__global__ void role_kernel(DevCSR g, const uint32_t *filler, uint32_t kind, uint32_t n_arg, uint32_t *out,
                            uint32_t n, uint32_t n_words, uint32_t wp) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wg * 32u < wp; wg += warps) {
        uint32_t v[1];
        role_words<1, 8>(g, filler, kind, n_arg, n, n_words, wg * 32u, lane, v);
        if (wg * 32u + lane < wp) out[wg * 32u + lane] = v[0];
    }
}

// A numeric or string concrete-role restriction (existential over each
// subject's values).
__global__ void exist_kernel(const uint32_t *rp, const uint32_t *vals, ValueTest test, uint32_t *out, uint32_t n,
                             uint32_t n_words, uint32_t wp) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wg * 32u < wp; wg += warps) {
        uint32_t v[1];
        exist_words<1>(rp, vals, test, n, n_words, wg * 32u, lane, v);
        if (wg * 32u + lane < wp) out[wg * 32u + lane] = v[0];
    }
}

__global__ void data_kernel(const float *vals, uint32_t cmp, float t, uint32_t *out, uint32_t n, uint32_t n_words,
                            uint32_t wp) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wg * 32u < wp; wg += warps) {
        uint32_t v[1];
        data_words<1>(vals, cmp, t, n, n_words, wg * 32u, lane, v);
        if (wg * 32u + lane < wp) out[wg * 32u + lane] = v[0];
    }
}

// Coverage count of one instance set: TP = |R & P|, FP = |R & N|
// (Algorithm 15), warp-reduced, one atomic pair per warp.
__global__ void score_kernel(const uint32_t *__restrict__ r, const uint32_t *__restrict__ pos,
                             const uint32_t *__restrict__ neg, uint32_t wp, uint32_t *acc) {
    uint32_t tp = 0, fp = 0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < wp / 4; q += gridDim.x * blockDim.x) {
        const uint4 a = *reinterpret_cast<const uint4 *>(r + 4 * q);
        const uint4 p = __ldg(reinterpret_cast<const uint4 *>(pos + 4 * q));
        const uint4 m = __ldg(reinterpret_cast<const uint4 *>(neg + 4 * q));
        tp += __popc(a.x & p.x) + __popc(a.y & p.y) + __popc(a.z & p.z) + __popc(a.w & p.w);
        fp += __popc(a.x & m.x) + __popc(a.y & m.y) + __popc(a.z & m.z) + __popc(a.w & m.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tp += __shfl_xor_sync(FULL, tp, o);
        fp += __shfl_xor_sync(FULL, fp, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        if (tp) atomicAdd(acc, tp);
        if (fp) atomicAdd(acc + 1, fp);
    }
}

__global__ void plain_finalize(KBView kb, const uint32_t *acc, uint32_t H, uint32_t *counts) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < H; h += gridDim.x * blockDim.x) {
        const uint32_t tp = acc[2 * h], fp = acc[2 * h + 1];
        *reinterpret_cast<uint4 *>(counts + 4ull * h) = make_uint4(tp, fp, kb.n_pos - tp, kb.n_neg - fp);
    }
}

uint32_t grid_for(uint64_t units, uint32_t per_block, int n_sms) {
    uint64_t g = (units + per_block - 1) / per_block;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(g, (uint64_t)n_sms * 8));
}

}  // namespace

int launch_plain(const hedl_kb *kb, const PlanImpl *p, uint32_t *counts, uint32_t *out_bits, void *ws,
                 void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const KBView v = kb->view();
    const uint32_t wp = kb->wp, H = p->n_hyps;
    uint8_t *base = (uint8_t *)ws;
    uint32_t *acc = (uint32_t *)(base + 256);
    const uint64_t rows_off = (256 + 8ull * H + 255) & ~uint64_t(255);
    uint32_t *rows = (uint32_t *)(base + rows_off);
    const uint32_t n_rows = p->plain_depth + 1;
    cudaError_t e = cudaMemsetAsync(acc, 0, 8ull * H, s);
    if (e) return e;
    const uint32_t g_quad = grid_for(wp / 4, PT, kb->n_sms);
    const uint32_t g_warp = grid_for(wp / 32 + 1, PT / 32, kb->n_sms);

    struct Val { const uint32_t *ptr; int row; };  // row >= 0: a workspace row to give back
    std::vector<Val> st;
    std::vector<int> free_rows;
    for (int r = (int)n_rows - 1; r >= 0; --r) free_rows.push_back(r);
    auto take = [&]() { int r = free_rows.back(); free_rows.pop_back(); return r; };
    auto give = [&](const Val &x) { if (x.row >= 0) free_rows.push_back(x.row); };
    auto row_ptr = [&](int r) { return rows + (uint64_t)r * wp; };

    for (uint32_t h = 0; h < H; ++h) {
        st.clear();
        for (uint32_t k = p->offs[h]; k < p->offs[h + 1]; ++k) {
            const uint64_t w = p->progs[k];
            const uint32_t op = (uint32_t)(w & 0xFF), inv = (uint32_t)((w >> 8) & 1);
            const uint32_t a = (uint32_t)((w >> 16) & 0xFFFF), b = (uint32_t)(w >> 32);
            if (op == HEDL_OP_ATOM) {  // read in place, as the paper's kernels read the concepts matrix
                st.push_back({kb->concepts + (uint64_t)a * wp, -1});
                continue;
            }
            const int r = take();
            uint32_t *out = row_ptr(r);
            if (op == HEDL_OP_TOP || op == HEDL_OP_BOT) {
                bool_kernel<<<g_quad, PT, 0, s>>>(op, nullptr, nullptr, out, wp, v.w, v.n);
            } else if (op == HEDL_OP_NOT) {
                Val x = st.back();
                st.pop_back();
                bool_kernel<<<g_quad, PT, 0, s>>>(op, x.ptr, nullptr, out, wp, v.w, v.n);
                give(x);
            } else if (op == HEDL_OP_AND || op == HEDL_OP_OR) {
                Val y = st.back();
                st.pop_back();
                Val x = st.back();
                st.pop_back();
                bool_kernel<<<g_quad, PT, 0, s>>>(op, x.ptr, y.ptr, out, wp, v.w, v.n);
                give(x);
                give(y);
            } else if (op == HEDL_OP_SEQ || op == HEDL_OP_SCONTAINS) {   // a string concrete role
                exist_kernel<<<g_warp, PT, 0, s>>>(kb->str_host[a].rp, kb->str_host[a].ids,
                                                   value_test(v, op << 16, b), out, v.n, v.w, wp);
            } else if (op >= HEDL_OP_DGE) {
                float t;
                memcpy(&t, &b, sizeof t);
                if (a >= kb->n_props) {   // a numeric concrete role
                    const DevNum &g = kb->num_host[a - kb->n_props];
                    exist_kernel<<<g_warp, PT, 0, s>>>(g.rp, reinterpret_cast<const uint32_t *>(g.vals),
                                                       value_test(v, op << 16, b), out, v.n, v.w, wp);
                } else {
                    data_kernel<<<g_warp, PT, 0, s>>>(kb->props + (uint64_t)a * kb->prop_stride, op, t, out, v.n,
                                                      v.w, wp);
                }
            } else {  // role restriction
                Val x = st.back();
                st.pop_back();
                role_kernel<<<g_warp, PT, 0, s>>>(kb->csr_host[2 * a + inv], x.ptr, op, b, out, v.n, v.w, wp);
                give(x);
            }
            st.push_back({out, r});
            e = cudaGetLastError();
            if (e) return e;
        }
        const Val res = st.back();
        if (out_bits) {
            e = cudaMemcpyAsync(out_bits + (uint64_t)h * wp, res.ptr, 4ull * wp, cudaMemcpyDeviceToDevice, s);
            if (e) return e;
        }
        if (counts) score_kernel<<<g_quad, PT, 0, s>>>(res.ptr, kb->pos, kb->neg, wp, acc + 2 * h);
        give(res);
        e = cudaGetLastError();
        if (e) return e;
    }
    if (counts) plain_finalize<<<grid_for(H, PT, kb->n_sms), PT, 0, s>>>(v, acc, H, counts);
    return cudaGetLastError();
}

}  // namespace hedl
