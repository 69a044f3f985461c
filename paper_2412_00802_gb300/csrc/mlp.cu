// The learned surrogate: structural encoder, a 512-512-512-2 MLP with BF16
// weights/activations and FP32 accumulation (forward, backward, Adam), exact
// scores from coverage counts, and a deterministic top-k selection.  The
// paper has no counterpart; the surrogate only orders and prunes the queue of
// exact evaluations.
//
// The dense layers run on the tensor cores through a warp-level BF16 GEMM
// (mma.sync m16n8k16, operands staged in shared memory and read with
// ldmatrix, FP32 accumulators in registers) with fused epilogues: bias, ReLU,
// the ReLU-derivative mask of the backward pass, BF16 or FP32 output, and a
// split-K mode that accumulates weight gradients with atomics.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "hedl_internal.h"

namespace hedl {
namespace {

constexpr int DI = 512, DH = 512, DO = 2;

// ------------------------------------------------------------------ encoder
__device__ __forceinline__ int arity_of(uint32_t op) {
    if (op == HEDL_OP_NOT || (op >= HEDL_OP_EXISTS && op <= HEDL_OP_EXACTLY)) return 1;
    if (op == HEDL_OP_AND || op == HEDL_OP_OR) return 2;
    return 0;
}

constexpr int ENC_MAXLEN = 256;

// One warp per program: lane 0 computes node depths and polarities (a
// reversed walk of the postfix is a pre-order walk; NOT and ATMOST flip the
// polarity of their operand), then the lanes count features into shared
// memory and write the row as bf16 (counts x 1/4, exact), the two prior
// inputs as bf16 of the caller's values.  Signed counts add +1 at polarity 0
// and -1 at polarity 1.
//   [  0, 84) op x min(depth, 5)          [ 84,180) concept mod 96, signed
//   [180,244) role mod 32 x inverse       [244,284) restriction kind x depth
//   [284,308) cardinality                 [308,436) property mod 16 x (>=, <=) x bucket / 4, signed
//   [436,493) role-over-atom hash mod 57, signed
//   [493,497) length / 10                 [497,504) statistics sums, signed
//   [504,510) totals, height, constant    [510,512) prior
// stats (or null): n_sc atom scores, then n_grid x 2 x 16 threshold scores.
__global__ void encode_kernel(const uint64_t *__restrict__ progs, const uint32_t *__restrict__ offs, uint32_t H,
                              const float *__restrict__ grid, uint32_t n_grid, const int32_t *__restrict__ stats,
                              uint32_t n_sc, const float *__restrict__ prior, __nv_bfloat16 *__restrict__ X) {
    constexpr int WARPS = 4;
    __shared__ int feat[WARPS][DI];
    __shared__ uint8_t depth[WARPS][ENC_MAXLEN];
    __shared__ uint8_t pol[WARPS][ENC_MAXLEN];
    __shared__ uint8_t pend[WARPS][ENC_MAXLEN + 1];    // pending depth (7 bits) | polarity << 7
    __shared__ uint32_t height[WARPS];
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint32_t h = blockIdx.x * WARPS + warp; h < H; h += gridDim.x * WARPS) {
        for (int i = lane; i < DI; i += 32) feat[warp][i] = 0;
        // programs longer than ENC_MAXLEN are encoded by their last ENC_MAXLEN
        // instructions (the root and the nodes nearest to it)
        const uint32_t L = min(offs[h + 1] - offs[h], (uint32_t)ENC_MAXLEN), o0 = offs[h + 1] - L;
        if (lane == 0) {
            int sp = 0;
            pend[warp][sp++] = 0;
            uint32_t ht = 0;
            for (int k = (int)L - 1; k >= 0; --k) {
                if (sp == 0) {   // not a well-formed program: remaining nodes get depth 0, polarity 0
                    for (; k >= 0; --k) depth[warp][k] = 0, pol[warp][k] = 0;
                    break;
                }
                const uint32_t e = pend[warp][--sp];
                const uint32_t d = e & 0x7Fu, pl = e >> 7;
                depth[warp][k] = (uint8_t)d;
                pol[warp][k] = (uint8_t)pl;
                ht = max(ht, d + 1);
                const uint32_t op = (uint32_t)(progs[o0 + k] & 0xFF);
                const int a = arity_of(op);
                // depths beyond 127 only feed clamped features (depth 7, height 8)
                const uint32_t flip = (op == HEDL_OP_NOT || op == HEDL_OP_ATMOST) ? 1u : 0u;
                const uint32_t ce = min(d + 1, 127u) | ((pl ^ flip) << 7);
                for (int j = 0; j < a && sp <= ENC_MAXLEN; ++j) pend[warp][sp++] = (uint8_t)ce;
            }
            height[warp] = ht;
        }
        __syncwarp();
        for (uint32_t k = lane; k < L; k += 32) {
            const uint64_t w = progs[o0 + k];
            const uint32_t op = (uint32_t)(w & 0xFF), inv = (uint32_t)((w >> 8) & 1);
            const uint32_t a = (uint32_t)((w >> 16) & 0xFFFF), b = (uint32_t)(w >> 32);
            if (op < HEDL_OP_ATOM || op > HEDL_OP_DEQ) continue;   // no feature: not an op, or a string restriction
            const uint32_t dk = depth[warp][k];
            const int sign = pol[warp][k] ? -1 : 1;
            atomicAdd(&feat[warp][min(dk, 5u) * 14 + op - 1], 1);
            if (arity_of(op) == 0) atomicAdd(&feat[warp][504], 1);
            if (op == HEDL_OP_ATOM) {
                atomicAdd(&feat[warp][84 + a % 96], sign);
                if (stats && a < n_sc) atomicAdd(&feat[warp][497 + min(dk / 2, 2u)], sign * stats[a]);
            } else if (op >= HEDL_OP_EXISTS && op <= HEDL_OP_EXACTLY) {
                atomicAdd(&feat[warp][505], 1);
                atomicAdd(&feat[warp][180 + (a % 32) * 2 + inv], 1);
                atomicAdd(&feat[warp][244 + min(dk, 7u) * 5 + (op - HEDL_OP_EXISTS)], 1);
                if (op >= HEDL_OP_ATLEAST) atomicAdd(&feat[warp][284 + (op - HEDL_OP_ATLEAST) * 8 + min(b, 7u)], 1);
                if (k > 0) {   // the filler ends right before its restriction
                    const uint64_t c = progs[o0 + k - 1];
                    if ((c & 0xFF) == HEDL_OP_ATOM) {
                        const uint32_t cc = (uint32_t)((c >> 16) & 0xFFFF);
                        atomicAdd(&feat[warp][436 + ((a * 2 + inv) * 131 + cc) % 57], sign);
                        if (stats && cc < n_sc) atomicAdd(&feat[warp][503], sign * stats[cc]);
                    }
                }
            } else if (op >= HEDL_OP_DGE) {
                atomicAdd(&feat[warp][506], 1);
                if (op != HEDL_OP_DEQ) {
                    const float t = __uint_as_float(b);
                    uint32_t q = 0;
                    if (grid && a < n_grid && !(t != t))
                        for (int g = 0; g < 15; ++g) q += grid[a * 15 + g] < t ? 1u : 0u;
                    atomicAdd(&feat[warp][308 + ((a % 16) * 2 + (op - HEDL_OP_DGE)) * 4 + q / 4], sign);
                    if (stats && a < n_grid)
                        atomicAdd(&feat[warp][500 + min(dk / 2, 2u)],
                                  sign * stats[n_sc + (a * 2 + (op - HEDL_OP_DGE)) * 16 + q]);
                }
            } else if (op == HEDL_OP_NOT) {
                atomicAdd(&feat[warp][507], 1);
            }
        }
        __syncwarp();
        if (lane == 0) {
            feat[warp][493 + min(L, 39u) / 10] += 1;
            feat[warp][508] += (int)min(height[warp], 8u) - 1;
            feat[warp][509] += 4;
        }
        __syncwarp();
        for (int i = lane; i < DI; i += 32) {
            __nv_bfloat16 x;
            if (i >= DI - 2) x = __float2bfloat16_rn(prior ? prior[2ull * h + (i - (DI - 2))] : 0.0f);
            else x = __float2bfloat16_rn(0.25f * (float)feat[warp][i]);
            X[(uint64_t)h * DI + i] = x;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ tensor-core GEMM
// C[M,N] = sum_k A(m,k) B(k,n), A and B bf16, FP32 accumulation.
//   A_KM: A stored [K][M] (else [M][K]);  B_KN: B stored [K][N] (else [N][K]).
// Tiles: 128 x 128 x 32, 8 warps of 64 x 32, mma.sync.m16n8k16.
constexpr int BM = 128, BN = 128, BK = 32, PAD = 8;

struct GemmArgs {
    const __nv_bfloat16 *A;
    const __nv_bfloat16 *B;
    void *C;
    const float *bias;              // [N] or null
    const __nv_bfloat16 *mask;      // [M][N] (ld = ldc): keep where mask > 0, or null
    int M, N, K, lda, ldb, ldc;
    int relu, out_bf16, atomic;     // atomic: FP32 atomicAdd into C (split-K)
    int k_chunk;                    // K range per blockIdx.z
};

__device__ __forceinline__ void ldsm_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(a));
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Load a 128 x 32 operand tile into smem as [row][k] (k contiguous); rows are
// M (or N) indices.  KMAJ: the operand is stored [rows][K]; else [K][rows].
template <bool KMAJ>
__device__ __forceinline__ void load_tile(__nv_bfloat16 (*dst)[BK + PAD], const __nv_bfloat16 *src, int rows,
                                          int K, int ld, int r0, int k0) {
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    if constexpr (KMAJ) {
        for (int idx = threadIdx.x; idx < BM * (BK / 8); idx += blockDim.x) {
            const int r = idx / (BK / 8), kc = (idx % (BK / 8)) * 8;
            const int gr = r0 + r, gk = k0 + kc;
            __nv_bfloat16 *d = &dst[r][kc];
            const __nv_bfloat16 *s = src + (size_t)gr * ld + gk;
            if (gr < rows && gk + 8 <= K && ((reinterpret_cast<uintptr_t>(s) & 15) == 0)) {
                *reinterpret_cast<uint4 *>(d) = *reinterpret_cast<const uint4 *>(s);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) d[j] = (gr < rows && gk + j < K) ? s[j] : zero;
            }
        }
    } else {
        for (int idx = threadIdx.x; idx < BK * (BM / 8); idx += blockDim.x) {
            const int k = idx / (BM / 8), rc = (idx % (BM / 8)) * 8;
            const int gk = k0 + k, gr = r0 + rc;
            const __nv_bfloat16 *s = src + (size_t)gk * ld + gr;
            __nv_bfloat16 v[8];
            if (gk < K && gr + 8 <= rows && ((reinterpret_cast<uintptr_t>(s) & 15) == 0)) {
                *reinterpret_cast<uint4 *>(v) = *reinterpret_cast<const uint4 *>(s);
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = (gk < K && gr + j < rows) ? s[j] : zero;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) dst[rc + j][k] = v[j];
        }
    }
}

template <bool A_KM, bool B_KN>
__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp >> 2, wn = warp & 3;          // 2 x 4 warps
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * g.k_chunk, ke = min(g.K, kb + g.k_chunk);
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += BK) {
        // operands restricted to this split's K range
        load_tile<!A_KM>(As, g.A, g.M, ke, g.lda, m0, k0);
        load_tile<!B_KN>(Bs, g.B, g.N, ke, g.ldb, n0, k0);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[4][4];
#pragma unroll
            for (int mt = 0; mt < 4; ++mt) {
                const int r = wm * 64 + mt * 16 + (lane & 15), c = kk + (lane >> 4) * 8;
                ldsm_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3], &As[r][c]);
            }
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                uint32_t b0, b1, b2, b3;
                const int r = wn * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3);
                const int c = kk + ((lane >> 3) & 1) * 8;
                ldsm_x4(b0, b1, b2, b3, &Bs[r][c]);
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    mma16816(acc[mt][np * 2 + 0], af[mt], b0, b1);
                    mma16816(acc[mt][np * 2 + 1], af[mt], b2, b3);
                }
            }
        }
        __syncthreads();
    }
    // epilogue
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int row = m0 + wm * 64 + mt * 16 + (lane >> 2) + half * 8;
                const int col = n0 + wn * 32 + nt * 8 + (lane & 3) * 2;
                if (row >= g.M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int cc = col + e;
                    if (cc >= g.N) continue;
                    float v = acc[mt][nt][half * 2 + e];
                    if (g.bias) v += g.bias[cc];
                    if (g.relu) v = fmaxf(v, 0.f);
                    if (g.mask && !(__bfloat162float(g.mask[(size_t)row * g.ldc + cc]) > 0.f)) v = 0.f;
                    if (g.atomic) atomicAdd(reinterpret_cast<float *>(g.C) + (size_t)row * g.ldc + cc, v);
                    else if (g.out_bf16)
                        reinterpret_cast<__nv_bfloat16 *>(g.C)[(size_t)row * g.ldc + cc] = __float2bfloat16_rn(v);
                    else reinterpret_cast<float *>(g.C)[(size_t)row * g.ldc + cc] = v;
                }
            }
}

int gemm(const GemmArgs &a0, bool a_km, bool b_kn, int splits, cudaStream_t s) {
    GemmArgs a = a0;
    splits = std::max(1, splits);
    a.k_chunk = ((a.K + splits - 1) / splits + BK - 1) / BK * BK;
    dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, (a.K + a.k_chunk - 1) / a.k_chunk);
    if (a_km && b_kn) gemm_kernel<true, true><<<grid, 256, 0, s>>>(a);
    else if (a_km) gemm_kernel<true, false><<<grid, 256, 0, s>>>(a);
    else if (b_kn) gemm_kernel<false, true><<<grid, 256, 0, s>>>(a);
    else gemm_kernel<false, false><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ output layer (N = 2)
// Y[b][j] = sum_i H2[b][i] W3[j][i] + b3[j]: one warp per row.
// With map (DEVICE float[5]: mean0, mean1, scale0, scale1, tail weight), the
// raw output u is mapped back to the target scale: Y = u * scale + mean.
// y = (u + b3), mapped back to the target scale when map is set, from the
// fused output layer's sums u (the unfused path's out_fwd_kernel semantics).
__global__ void out_map_kernel(const float *u, const float *b3, float *Y, int B, const float *map) {
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < B; row += gridDim.x * blockDim.x) {
        float u0 = u[2 * row] + b3[0], u1 = u[2 * row + 1] + b3[1];
        if (map) {
            u0 = u0 * map[2] + map[0];
            u1 = u1 * map[3] + map[1];
        }
        Y[2 * row] = u0;
        Y[2 * row + 1] = u1;
    }
}

__global__ void out_fwd_kernel(const __nv_bfloat16 *H2, const __nv_bfloat16 *W3, const float *b3, float *Y, int B,
                               const float *map) {
    // warp per row (grid-stride); lane l holds columns 16l .. 16l+15 of both W3 rows
    const int lane = threadIdx.x & 31;
    float w0[16], w1[16];
    {
        const uint4 *p0 = reinterpret_cast<const uint4 *>(W3 + 16 * lane);
        const uint4 *p1 = reinterpret_cast<const uint4 *>(W3 + DH + 16 * lane);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint4 a = p0[q], c = p1[q];
            const uint32_t av[4] = {a.x, a.y, a.z, a.w}, cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 x = *reinterpret_cast<const __nv_bfloat162 *>(&av[e]);
                const __nv_bfloat162 y = *reinterpret_cast<const __nv_bfloat162 *>(&cv[e]);
                w0[q * 8 + 2 * e] = __low2float(x), w0[q * 8 + 2 * e + 1] = __high2float(x);
                w1[q * 8 + 2 * e] = __low2float(y), w1[q * 8 + 2 * e + 1] = __high2float(y);
            }
        }
    }
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < B; row += warps) {
        const uint4 *h = reinterpret_cast<const uint4 *>(H2 + (size_t)row * DH + 16 * lane);
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const uint4 a = h[q];
            const uint32_t av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 x = *reinterpret_cast<const __nv_bfloat162 *>(&av[e]);
                const float lo = __low2float(x), hi = __high2float(x);
                s0 += lo * w0[q * 8 + 2 * e] + hi * w0[q * 8 + 2 * e + 1];
                s1 += lo * w1[q * 8 + 2 * e] + hi * w1[q * 8 + 2 * e + 1];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, o);
            s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
        }
        if (lane == 0) {
            float u0 = s0 + b3[0], u1 = s1 + b3[1];
            if (map) {
                u0 = u0 * map[2] + map[0];
                u1 = u1 * map[3] + map[1];
            }
            Y[2 * row] = u0;
            Y[2 * row + 1] = u1;
        }
    }
}

// Raw outputs U against mapped targets t' = (T - mean) / scale, row weight
// w = 1 + tail * max(0, t'_0) (the upper tail of the first target counts
// more): dU = 2 w (U - t') / B; loss += w (U - t')^2 / B.
__global__ void loss_kernel(const float *U, const float *T, float *dU, float *loss, int B, const float *map) {
    float l = 0.f;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        const float t0 = (T[2 * b] - map[0]) / map[2], t1 = (T[2 * b + 1] - map[1]) / map[3];
        const float w = 1.f + map[4] * fmaxf(t0, 0.f);
        const float d0 = U[2 * b] - t0, d1 = U[2 * b + 1] - t1;
        dU[2 * b] = 2.f * w * d0 / (float)B;
        dU[2 * b + 1] = 2.f * w * d1 / (float)B;
        l += w * (d0 * d0 + d1 * d1) / (float)B;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// Target map from a target set: column means, column standard deviations
// (population; 1 where below 1e-6), the tail weight.  One block, float64 sums.
__global__ void fit_map_kernel(const float *T, int B, float tail, float *map) {
    __shared__ double red[2][1024];
    double s0 = 0, s1 = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s0 += T[2 * b], s1 += T[2 * b + 1];
    red[0][threadIdx.x] = s0, red[1][threadIdx.x] = s1;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[0][threadIdx.x] += red[0][threadIdx.x + o], red[1][threadIdx.x] += red[1][threadIdx.x + o];
        __syncthreads();
    }
    const double m0 = red[0][0] / B, m1 = red[1][0] / B;
    __syncthreads();
    double v0 = 0, v1 = 0;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const double d0 = T[2 * b] - m0, d1 = T[2 * b + 1] - m1;
        v0 += d0 * d0, v1 += d1 * d1;
    }
    red[0][threadIdx.x] = v0, red[1][threadIdx.x] = v1;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[0][threadIdx.x] += red[0][threadIdx.x + o], red[1][threadIdx.x] += red[1][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sd0 = sqrt(red[0][0] / B), sd1 = sqrt(red[1][0] / B);
        map[0] = (float)m0, map[1] = (float)m1;
        map[2] = sd0 < 1e-6 ? 1.f : (float)sd0;
        map[3] = sd1 < 1e-6 ? 1.f : (float)sd1;
        map[4] = tail;
    }
}

// dH2[b][i] = (dY[b][0] W3[0][i] + dY[b][1] W3[1][i]) * [H2[b][i] > 0]  (bf16)
__global__ void out_bwd_dh_kernel(const float *dY, const __nv_bfloat16 *W3, const __nv_bfloat16 *H2,
                                  __nv_bfloat16 *dH2, int B) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)B * DH;
         e += (size_t)gridDim.x * blockDim.x) {
        const size_t b = e / DH, i = e % DH;
        float v = dY[2 * b] * __bfloat162float(W3[i]) + dY[2 * b + 1] * __bfloat162float(W3[DH + i]);
        if (!(__bfloat162float(H2[e]) > 0.f)) v = 0.f;
        dH2[e] = __float2bfloat16_rn(v);
    }
}

// dW3[j][i] = sum_b dY[b][j] H2[b][i]; db3[j] = sum_b dY[b][j] (one thread per i, FP32)
__global__ void out_bwd_dw_kernel(const float *dY, const __nv_bfloat16 *H2, float *dW3, float *db3, int B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < DH) {
        float s0 = 0.f, s1 = 0.f;
        for (int b = 0; b < B; ++b) {
            const float h = __bfloat162float(H2[(size_t)b * DH + i]);
            s0 += dY[2 * b] * h;
            s1 += dY[2 * b + 1] * h;
        }
        dW3[i] = s0;
        dW3[DH + i] = s1;
    }
    if (i == 0) {
        float s0 = 0.f, s1 = 0.f;
        for (int b = 0; b < B; ++b) {
            s0 += dY[2 * b];
            s1 += dY[2 * b + 1];
        }
        db3[0] = s0;
        db3[1] = s1;
    }
}

// db[i] = sum_b dH[b][i]
__global__ void colsum_kernel(const __nv_bfloat16 *dH, float *db, int B, int D) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += __bfloat162float(dH[(size_t)b * D + i]);
    db[i] = s;
}

// Adam on FP32 master weights; refreshes the BF16 copy.
// dst[c][r] = src[r][c] for an R x C bf16 matrix (32 x 32 tiles through shared memory).
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *src, int R, int C, int lds, __nv_bfloat16 *dst, int ldd) {
    __shared__ __nv_bfloat16 t[32][34];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = src[(size_t)r * lds + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) dst[(size_t)c * ldd + r] = t[threadIdx.x][i];
    }
}

void transpose_bf16(const __nv_bfloat16 *src, int R, int C, int lds, __nv_bfloat16 *dst, int ldd, cudaStream_t s) {
    transpose_bf16_kernel<<<dim3((C + 31) / 32, (R + 31) / 32), dim3(32, 8), 0, s>>>(src, R, C, lds, dst, ldd);
}

__global__ void adam_kernel(float *w, float *m, float *v, const float *g, __nv_bfloat16 *wb, size_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        if (wb) wb[i] = __float2bfloat16_rn(wi);
    }
}

__global__ void to_bf16_kernel(const float *src, __nv_bfloat16 *dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

// accuracy = (TP + TN) / (|P| + |N|), F1 = 2TP / (2TP + FP + FN) (0 if the denominator is 0)
// Statistics table entries from exact scores: round((accuracy - 1/2) * 32), in double.
__global__ void stat_kernel(const float *scores, uint32_t n, int32_t *out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (int32_t)rint(((double)scores[2 * i] - 0.5) * 32.0);
}

__global__ void scores_kernel(const uint32_t *counts, uint32_t H, float *T) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < H; h += gridDim.x * blockDim.x) {
        const uint4 c = reinterpret_cast<const uint4 *>(counts)[h];
        const double tot = (double)c.x + c.y + c.z + c.w;
        const double den = 2.0 * c.x + c.y + c.z;
        T[2 * h] = tot > 0 ? (float)(((double)c.x + c.w) / tot) : 0.f;
        T[2 * h + 1] = den > 0 ? (float)(2.0 * c.x / den) : 0.f;
    }
}

// ------------------------------------------------------------------ top-k
// Key of a prediction for "larger is better" with ties broken by F1 then by
// smaller index: (accuracy bits, F1 bits) mapped to order-preserving uint32.
__device__ __forceinline__ uint32_t order_key(float x) {
    uint32_t u = __float_as_uint(x);
    if (x != x) return 0u;                      // NaN ranks last
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// A radix select over 64-bit keys (accuracy key << 32 | F1 key) finds the
// k-th largest key 8 bits at a time; a single-block stable compaction then
// picks every larger key and, among equal keys, the lowest indices.
__global__ void keys_kernel(const float *Y, uint32_t H, unsigned long long *keys) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < H; h += gridDim.x * blockDim.x)
        keys[h] = ((unsigned long long)order_key(Y[2 * h]) << 32) | order_key(Y[2 * h + 1]);
}

// One pass of the radix select: histogram of the 8 bits at `shift` among the
// keys whose bits above shift+8 equal the prefix chosen so far (*prefix).
__global__ void radix_hist_kernel(const unsigned long long *keys, uint32_t H, const unsigned long long *prefix,
                                  int shift, uint32_t *hist) {
    __shared__ uint32_t sh[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const unsigned long long pmask = shift >= 56 ? 0ull : ~((1ull << (shift + 8)) - 1ull);
    const unsigned long long pre = *prefix & pmask;
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < H; h += gridDim.x * blockDim.x) {
        const unsigned long long k = keys[h];
        if ((k & pmask) == pre) atomicAdd(&sh[(k >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// state[0..1] = prefix (64 bits), state[2] = k remaining; picks the bucket
// holding the k-th largest and narrows the prefix.
__global__ void radix_pick_kernel(uint32_t *hist, int shift, unsigned long long *state_prefix, uint32_t *state_k) {
    if (threadIdx.x != 0) return;
    uint32_t k = *state_k;
    for (int b = 255; b >= 0; --b) {
        if (hist[b] >= k) {
            *state_prefix |= ((unsigned long long)b << shift);
            break;
        }
        k -= hist[b];
    }
    *state_k = k;
    for (int b = 0; b < 256; ++b) hist[b] = 0;
}

// Stable selection: every key > thr, then the first `ties` keys == thr in
// index order; output sorted by index.  One block, chunked prefix sums.
__global__ void select_kernel(const unsigned long long *keys, uint32_t H, const unsigned long long *thr_p,
                              const uint32_t *ties_p, uint32_t *out) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t base_gt, base_eq;
    const unsigned long long thr = *thr_p;
    const uint32_t ties = *ties_p;
    if (threadIdx.x == 0) base_gt = base_eq = 0;
    __syncthreads();
    // output in index order: a picked key's position is (#greater before it) + min(#equal before it, ties)
    for (uint32_t c0 = 0; c0 < H; c0 += blockDim.x) {
        const uint32_t h = c0 + threadIdx.x;
        const unsigned long long k = h < H ? keys[h] : 0ull;
        const uint32_t gt = (h < H && k > thr) ? 1u : 0u;
        const uint32_t eq = (h < H && k == thr) ? 1u : 0u;
        // block-wide exclusive scans of gt and eq (packed 16/16 bits per chunk of <= 1024)
        uint32_t v = gt | (eq << 16);
        const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= (uint32_t)o) incl += t;
        }
        if (lane == 31) warp_sums[w] = incl;
        __syncthreads();
        if (w == 0) {
            const uint32_t nw = (blockDim.x + 31) / 32;
            uint32_t x = lane < nw ? warp_sums[lane] : 0u;
            uint32_t y = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, y, o);
                if (lane >= (uint32_t)o) y += t;
            }
            if (lane < nw) warp_sums[lane] = y - x;   // exclusive per warp
        }
        __syncthreads();
        const uint32_t excl = incl - v + warp_sums[w];
        const uint32_t gt_before = base_gt + (excl & 0xFFFF), eq_before = base_eq + (excl >> 16);
        if (gt) out[gt_before + min(eq_before, ties)] = h;
        if (eq && eq_before < ties) out[gt_before + eq_before] = h;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
            base_gt += ((excl + v) & 0xFFFF);
            base_eq += ((excl + v) >> 16);
        }
        __syncthreads();
    }
}

}  // namespace
}  // namespace hedl

using namespace hedl;

struct hedl_mlp {
    // FP32 master weights, Adam moments, gradients; BF16 copies for compute;
    // the target map (mean0, mean1, scale0, scale1, tail weight)
    float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *map = nullptr;
    uint32_t *err = nullptr;                  // device: bit 0 = a tensor-core wait timed out
    __nv_bfloat16 *w2t = nullptr;             // W2 transposed ([in][out], bf16) for the backward GEMM
    unsigned gemm = HEDL_GEMM_TCGEN05;        // engine of the dense layers' forward GEMMs
    __nv_bfloat16 *wb = nullptr;
    size_t n = 0;
    uint32_t step = 0;
};

namespace {

constexpr size_t OFF_W1 = 0, OFF_B1 = OFF_W1 + (size_t)DH * DI, OFF_W2 = OFF_B1 + DH, OFF_B2 = OFF_W2 + (size_t)DH * DH,
                 OFF_W3 = OFF_B2 + DH, OFF_B3 = OFF_W3 + (size_t)DO * DH, N_PARAMS = OFF_B3 + DO;

struct MlpWs {
    __nv_bfloat16 *h1, *h2, *dh1, *dh2;
    float *y, *dy, *loss;
    __nv_bfloat16 *t0, *t1;   // transposed operands ([512][B]) of the tensor-core weight gradients
};

size_t mlp_ws_bytes(uint32_t B) { return 6 * (size_t)B * DH * 2 + 2 * (size_t)B * DO * 4 + 256 + 7 * 256; }

MlpWs carve(void *ws, uint32_t B) {
    uint8_t *p = (uint8_t *)ws;
    auto take = [&](size_t bytes) {
        uint8_t *r = p;
        p += (bytes + 255) & ~size_t(255);
        return r;
    };
    MlpWs w;
    w.h1 = (__nv_bfloat16 *)take((size_t)B * DH * 2);
    w.h2 = (__nv_bfloat16 *)take((size_t)B * DH * 2);
    w.dh1 = (__nv_bfloat16 *)take((size_t)B * DH * 2);
    w.dh2 = (__nv_bfloat16 *)take((size_t)B * DH * 2);
    w.y = (float *)take((size_t)B * DO * 4);
    w.dy = (float *)take((size_t)B * DO * 4);
    w.loss = (float *)take(4);
    w.t0 = (__nv_bfloat16 *)take((size_t)B * DH * 2);
    w.t1 = (__nv_bfloat16 *)take((size_t)B * DH * 2);
    return w;
}

uint32_t grid1(size_t n) { return (uint32_t)std::min<size_t>((n + 255) / 256, 4096); }

// One hidden layer, H = relu(A . W^T + b): on tcgen05 when selected (and the
// shape allows it), else on the mma.sync GEMM.
int dense_relu(hedl_mlp *mlp, const __nv_bfloat16 *A, const __nv_bfloat16 *W, const float *b, __nv_bfloat16 *H,
               int M, int K, cudaStream_t s) {
    UmmaArgs u{A, W, H, b, M, DH, K, K, K, DH, 1, 1, mlp->err, nullptr};
    if (mlp->gemm == HEDL_GEMM_TCGEN05 && umma_shape_ok(u)) return umma_gemm(u, s);
    GemmArgs a{};
    a.A = A;
    a.B = W;
    a.C = H;
    a.bias = b;
    a.M = M, a.N = DH, a.K = K, a.lda = K, a.ldb = K, a.ldc = DH;
    a.relu = 1, a.out_bf16 = 1;
    return gemm(a, false, false, 1, s);
}

int forward_impl(hedl_mlp *mlp, const __nv_bfloat16 *X, uint32_t B, const MlpWs &w, cudaStream_t s,
                 bool mapped, bool need_h2 = true) {
    int e = dense_relu(mlp, X, mlp->wb + OFF_W1, mlp->w + OFF_B1, w.h1, (int)B, DI, s);
    if (e) return e;
    if (!need_h2 && mlp->gemm == HEDL_GEMM_TCGEN05) {
        // inference: the second layer's epilogue computes the output layer (h2 is never written)
        UmmaArgs u{w.h1, mlp->wb + OFF_W2, w.h2, mlp->w + OFF_B2, (int)B, DH, DH, DH, DH, DH, 1, 1, mlp->err, nullptr};
        u.w3 = mlp->wb + OFF_W3;
        u.y = w.dy;   // [B][2] sums, zeroed first
        u.store = 0;
        if (umma_shape_ok(u)) {
            e = cudaMemsetAsync(w.dy, 0, (size_t)B * DO * 4, s);
            if (e) return e;
            e = umma_gemm(u, s);
            if (e) return e;
            out_map_kernel<<<std::min<uint32_t>((B + 255) / 256, 148u * 8u), 256, 0, s>>>(
                w.dy, mlp->w + OFF_B3, w.y, (int)B, mapped ? mlp->map : nullptr);
            return cudaGetLastError();
        }
    }
    e = dense_relu(mlp, w.h1, mlp->wb + OFF_W2, mlp->w + OFF_B2, w.h2, (int)B, DH, s);
    if (e) return e;
    out_fwd_kernel<<<std::min<uint32_t>((B * 32 + 255) / 256, 148u * 8u), 256, 0, s>>>(
        w.h2, mlp->wb + OFF_W3, mlp->w + OFF_B3, w.y, (int)B, mapped ? mlp->map : nullptr);
    return cudaGetLastError();
}

int grads_impl(hedl_mlp *mlp, const __nv_bfloat16 *X, const float *T, uint32_t B, const MlpWs &w, cudaStream_t s) {
    int e = forward_impl(mlp, X, B, w, s, false);
    if (e) return e;
    e = cudaMemsetAsync(w.loss, 0, 4, s);
    if (e) return e;
    e = cudaMemsetAsync(mlp->g, 0, N_PARAMS * 4, s);
    if (e) return e;
    loss_kernel<<<grid1(B), 256, 0, s>>>(w.y, T, w.dy, w.loss, (int)B, mlp->map);
    out_bwd_dw_kernel<<<(DH + 255) / 256, 256, 0, s>>>(w.dy, w.h2, mlp->g + OFF_W3, mlp->g + OFF_B3, (int)B);
    out_bwd_dh_kernel<<<grid1((size_t)B * DH), 256, 0, s>>>(w.dy, mlp->wb + OFF_W3, w.h2, w.dh2, (int)B);
    colsum_kernel<<<(DH + 255) / 256, 256, 0, s>>>(w.dh2, mlp->g + OFF_B2, (int)B, DH);
    if (mlp->gemm == HEDL_GEMM_TCGEN05 && B % 64 == 0) {
        // Weight gradients dW = dH^T . H on tcgen05 as K-major products over the
        // batch: both operands are transposed to [512][B] first.
        transpose_bf16(w.dh2, (int)B, DH, DH, w.t0, (int)B, s);
        transpose_bf16(w.h1, (int)B, DH, DH, w.t1, (int)B, s);
        UmmaArgs u{w.t0, w.t1, mlp->g + OFF_W2, nullptr, DH, DH, (int)B, (int)B, (int)B, DH, 0, 0, mlp->err,
                   nullptr};
        e = umma_gemm(u, s);
        if (e) return e;
        // dH1 = (dH2 . W2) * [H1 > 0], with W2 kept transposed ([in][out], K-major)
        UmmaArgs d{w.dh2, mlp->w2t, w.dh1, nullptr, (int)B, DH, DH, DH, DH, DH, 0, 1, mlp->err, w.h1};
        e = umma_gemm(d, s);
        if (e) return e;
        colsum_kernel<<<(DH + 255) / 256, 256, 0, s>>>(w.dh1, mlp->g + OFF_B1, (int)B, DH);
        transpose_bf16(w.dh1, (int)B, DH, DH, w.t0, (int)B, s);
        transpose_bf16(X, (int)B, DI, DI, w.t1, (int)B, s);
        UmmaArgs x{w.t0, w.t1, mlp->g + OFF_W1, nullptr, DH, DI, (int)B, (int)B, (int)B, DI, 0, 0, mlp->err,
                   nullptr};
        e = umma_gemm(x, s);
        if (e) return e;
        return cudaGetLastError();
    }
    const int splits = std::max(1, std::min((int)(B / 256), 64));
    // dW2 = dH2^T H1   (M = out, N = in, K = batch): A stored [K][M], B stored [K][N]
    GemmArgs a{};
    a.A = w.dh2;
    a.B = w.h1;
    a.C = mlp->g + OFF_W2;
    a.M = DH, a.N = DH, a.K = (int)B, a.lda = DH, a.ldb = DH, a.ldc = DH;
    a.atomic = 1;
    e = gemm(a, true, true, splits, s);
    if (e) return e;
    // dH1 = (dH2 W2) * [H1 > 0]   (M = batch, N = in, K = out): A [M][K], B stored [K][N]
    GemmArgs d{};
    d.A = w.dh2;
    d.B = mlp->wb + OFF_W2;
    d.C = w.dh1;
    d.mask = w.h1;
    d.M = (int)B, d.N = DH, d.K = DH, d.lda = DH, d.ldb = DH, d.ldc = DH;
    d.out_bf16 = 1;
    e = gemm(d, false, true, 1, s);
    if (e) return e;
    colsum_kernel<<<(DH + 255) / 256, 256, 0, s>>>(w.dh1, mlp->g + OFF_B1, (int)B, DH);
    // dW1 = dH1^T X
    a.A = w.dh1;
    a.B = X;
    a.C = mlp->g + OFF_W1;
    a.N = DI, a.ldb = DI;
    e = gemm(a, true, true, splits, s);
    if (e) return e;
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int hedl_mlp_create(const float *params, hedl_mlp **out) {
    if (!out || !params) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    auto *m = new hedl_mlp();
    m->n = N_PARAMS;
    cudaError_t e = cudaMalloc(&m->w, N_PARAMS * 4);
    if (!e) e = cudaMalloc(&m->m, N_PARAMS * 4);
    if (!e) e = cudaMalloc(&m->v, N_PARAMS * 4);
    if (!e) e = cudaMalloc(&m->g, N_PARAMS * 4);
    if (!e) e = cudaMalloc(&m->wb, N_PARAMS * 2);
    if (!e) e = cudaMalloc(&m->map, 5 * 4);
    if (!e) e = cudaMalloc(&m->err, 4);
    if (!e) e = cudaMemset(m->err, 0, 4);
    if (!e) e = cudaMalloc(&m->w2t, (size_t)DH * DH * 2);
    if (!e) {
        const float ident[5] = {0.f, 0.f, 1.f, 1.f, 0.f};
        e = cudaMemcpy(m->map, ident, sizeof(ident), cudaMemcpyHostToDevice);
    }
    if (!e) e = cudaMemcpy(m->w, params, N_PARAMS * 4, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(m->m, 0, N_PARAMS * 4);
    if (!e) e = cudaMemset(m->v, 0, N_PARAMS * 4);
    if (!e) {
        to_bf16_kernel<<<grid1(N_PARAMS), 256>>>(m->w, m->wb, N_PARAMS);
        transpose_bf16(m->wb + OFF_W2, DH, DH, DH, m->w2t, DH, 0);
        e = cudaDeviceSynchronize();
    }
    if (e) {
        int rc = cuda_fail(e, "hedl_mlp_create");
        hedl_mlp_free(m);
        return rc;
    }
    *out = m;
    return HEDL_OK;
}

void hedl_mlp_free(hedl_mlp *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    cudaFree(m->w);
    cudaFree(m->m);
    cudaFree(m->v);
    cudaFree(m->g);
    cudaFree(m->wb);
    cudaFree(m->map);
    cudaFree(m->err);
    cudaFree(m->w2t);
    delete m;
}

uint64_t hedl_mlp_param_count(void) { return N_PARAMS; }

int hedl_mlp_get(const hedl_mlp *m, float *params, float *grads, uint32_t *step) {
    if (!m) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (!e && params) e = cudaMemcpy(params, m->w, N_PARAMS * 4, cudaMemcpyDeviceToHost);
    if (!e && grads) e = cudaMemcpy(grads, m->g, N_PARAMS * 4, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(e, "hedl_mlp_get");
    if (step) *step = m->step;
    return HEDL_OK;
}

int hedl_mlp_get_moments(const hedl_mlp *m, float *first, float *second) {
    if (!m) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaDeviceSynchronize();
    if (!e && first) e = cudaMemcpy(first, m->m, N_PARAMS * 4, cudaMemcpyDeviceToHost);
    if (!e && second) e = cudaMemcpy(second, m->v, N_PARAMS * 4, cudaMemcpyDeviceToHost);
    return e ? cuda_fail(e, "hedl_mlp_get_moments") : HEDL_OK;
}

int hedl_mlp_workspace_size(uint32_t B, size_t *bytes) {
    if (!bytes) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    *bytes = mlp_ws_bytes(B);
    return HEDL_OK;
}

int hedl_encode(const uint64_t *progs, const uint32_t *offs, uint32_t H, const float *grid, uint32_t n_grid,
                const int32_t *stats, uint32_t n_stat_concepts, const float *prior, uint16_t *X, hedl_stream s) {
    if (!progs || !offs || !X) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (stats && !grid && n_grid) return fail(HEDL_ERR_INVALID_ARG, "threshold statistics need the grid");
    if (H == 0) return HEDL_OK;
    encode_kernel<<<std::min<uint32_t>((H + 3) / 4, 8192), 128, 0, (cudaStream_t)s>>>(
        progs, offs, H, grid, grid ? n_grid : 0u, stats, stats ? n_stat_concepts : 0u, prior, (__nv_bfloat16 *)X);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "encode launch") : HEDL_OK;
}

int hedl_mlp_forward(hedl_mlp *m, const uint16_t *X, uint32_t B, float *Y, void *ws, size_t ws_bytes,
                     hedl_stream s) {
    if (!m || !X || !Y) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (!ws || ws_bytes < mlp_ws_bytes(B)) return fail(HEDL_ERR_WORKSPACE_TOO_SMALL, "MLP workspace too small");
    MlpWs w = carve(ws, B);
    int e = forward_impl(m, (const __nv_bfloat16 *)X, B, w, (cudaStream_t)s, true, false);
    if (e) return cuda_fail(e, "mlp forward");
    e = cudaMemcpyAsync(Y, w.y, (size_t)B * DO * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)s);
    return e ? cuda_fail(e, "mlp forward copy") : HEDL_OK;
}

int hedl_mlp_gradients(hedl_mlp *m, const uint16_t *X, const float *T, uint32_t B, float *loss, void *ws,
                       size_t ws_bytes, hedl_stream s) {
    if (!m || !X || !T) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (!ws || ws_bytes < mlp_ws_bytes(B)) return fail(HEDL_ERR_WORKSPACE_TOO_SMALL, "MLP workspace too small");
    MlpWs w = carve(ws, B);
    int e = grads_impl(m, (const __nv_bfloat16 *)X, T, B, w, (cudaStream_t)s);
    if (e) return cuda_fail(e, "mlp gradients");
    if (loss) {
        e = cudaMemcpyAsync(loss, w.loss, 4, cudaMemcpyDeviceToDevice, (cudaStream_t)s);
        if (e) return cuda_fail(e, "loss copy");
    }
    return HEDL_OK;
}

int hedl_mlp_train_step(hedl_mlp *m, const uint16_t *X, const float *T, uint32_t B, float lr, float *loss,
                        void *ws, size_t ws_bytes, hedl_stream s) {
    int e = hedl_mlp_gradients(m, X, T, B, loss, ws, ws_bytes, s);
    if (e) return e;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    adam_kernel<<<grid1(N_PARAMS), 256, 0, (cudaStream_t)s>>>(m->w, m->m, m->v, m->g, m->wb, N_PARAMS, lr, b1, b2,
                                                                1e-8f, c1, c2);
    transpose_bf16(m->wb + OFF_W2, DH, DH, DH, m->w2t, DH, (cudaStream_t)s);
    cudaError_t ce = cudaGetLastError();
    return ce ? cuda_fail(ce, "adam launch") : HEDL_OK;
}

int hedl_mlp_fit_target_map(hedl_mlp *m, const float *T, uint32_t B, float tail_weight, hedl_stream s) {
    if (!m || !T) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (B == 0) return fail(HEDL_ERR_INVALID_ARG, "empty target set");
    if (!(tail_weight >= 0.f)) return fail(HEDL_ERR_INVALID_ARG, "tail_weight must be >= 0");
    fit_map_kernel<<<1, 1024, 0, (cudaStream_t)s>>>(T, (int)B, tail_weight, m->map);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "fit map launch") : HEDL_OK;
}

int hedl_mlp_set_target_map(hedl_mlp *m, const float *map) {
    if (!m || !map) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (!(map[2] > 0.f) || !(map[3] > 0.f) || !(map[4] >= 0.f))
        return fail(HEDL_ERR_INVALID_ARG, "scales must be > 0 and the tail weight >= 0");
    cudaError_t e = cudaMemcpy(m->map, map, 5 * 4, cudaMemcpyHostToDevice);
    return e ? cuda_fail(e, "set map") : HEDL_OK;
}

int hedl_mlp_set_gemm(hedl_mlp *m, unsigned engine) {
    if (!m) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (engine != HEDL_GEMM_TCGEN05 && engine != HEDL_GEMM_MMA_SYNC)
        return fail(HEDL_ERR_INVALID_ARG, "engine must be HEDL_GEMM_TCGEN05 or HEDL_GEMM_MMA_SYNC");
    m->gemm = engine;
    return HEDL_OK;
}

int hedl_mlp_status(hedl_mlp *m, hedl_stream s) {
    if (!m) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)s);
    if (e) return cuda_fail(e, "stream synchronize");
    uint32_t st = 0;
    e = cudaMemcpy(&st, m->err, 4, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(e, "status read");
    if (st) {
        cudaMemset(m->err, 0, 4);
        return fail(HEDL_ERR_TIMEOUT, "a tensor-core completion wait gave up (timeout)");
    }
    return HEDL_OK;
}

int hedl_mlp_get_target_map(const hedl_mlp *m, float *map) {
    if (!m || !map) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaMemcpy(map, m->map, 5 * 4, cudaMemcpyDeviceToHost);
    return e ? cuda_fail(e, "get map") : HEDL_OK;
}

int hedl_stat_scores(const float *scores, uint32_t n, int32_t *out, hedl_stream s) {
    if (!scores || !out) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return HEDL_OK;
    stat_kernel<<<grid1(n), 256, 0, (cudaStream_t)s>>>(scores, n, out);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "stat launch") : HEDL_OK;
}

int hedl_scores_from_counts(const uint32_t *counts, uint32_t H, float *scores, hedl_stream s) {
    if (!counts || !scores) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (H == 0) return HEDL_OK;
    scores_kernel<<<grid1(H), 256, 0, (cudaStream_t)s>>>(counts, H, scores);
    cudaError_t e = cudaGetLastError();
    return e ? cuda_fail(e, "scores launch") : HEDL_OK;
}

int hedl_select_workspace_size(uint32_t H, size_t *bytes) {
    if (!bytes) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    *bytes = 8ull * H + 4096 + 256;
    return HEDL_OK;
}

int hedl_select_top(const float *Y, uint32_t H, uint32_t k, uint32_t *idx, void *ws, size_t ws_bytes,
                    hedl_stream s) {
    if (!Y || !idx) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (k == 0 || k > H) return fail(HEDL_ERR_INVALID_ARG, "k must be in 1..H");
    if (!ws || ws_bytes < 8ull * H + 4096 + 256) return fail(HEDL_ERR_WORKSPACE_TOO_SMALL, "select workspace too small");
    cudaStream_t st = (cudaStream_t)s;
    uint8_t *p = (uint8_t *)ws;
    auto *keys = (unsigned long long *)p;
    uint8_t *q = p + ((8ull * H + 255) & ~255ull);
    auto *hist = (uint32_t *)q;                          // 256 words
    auto *prefix = (unsigned long long *)(q + 1024);     // the k-th largest key, built 8 bits at a time
    auto *krem = (uint32_t *)(q + 1032);                 // rank still sought within the prefix
    cudaError_t e = cudaMemsetAsync(q, 0, 2048, st);
    if (!e) e = cudaMemcpyAsync(krem, &k, 4, cudaMemcpyHostToDevice, st);
    if (e) return cuda_fail(e, "select setup");
    keys_kernel<<<grid1(H), 256, 0, st>>>(Y, H, keys);
    for (int shift = 56; shift >= 0; shift -= 8) {
        radix_hist_kernel<<<grid1(H), 256, 0, st>>>(keys, H, prefix, shift, hist);
        radix_pick_kernel<<<1, 32, 0, st>>>(hist, shift, prefix, krem);
    }
    select_kernel<<<1, 1024, 0, st>>>(keys, H, prefix, krem, idx);
    e = cudaGetLastError();
    return e ? cuda_fail(e, "select launch") : HEDL_OK;
}

}  // extern "C"
