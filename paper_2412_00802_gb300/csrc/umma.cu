// Dense layer GEMM of the surrogate on the 5th-generation tensor cores:
// C[M][N] = act(A[M][K] . B[N][K]^T + bias), A and B bf16 and K-major (rows
// of K contiguous elements), FP32 accumulation in tensor memory (TMEM).
//
// A persistent kernel: one CTA per SM walks the 128 x 256 output tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Its six warps have fixed roles:
//   warp 0 (one thread): the TMA producer.  It loads each 64-wide K block of
//     the tile's A (128 x 64) and B (256 x 64) with one TMA copy each
//     (cp.async.bulk.tensor, 128-byte rows in the 128-byte swizzle the
//     tensor cores read as K-major SWIZZLE_128B operands) into a ring of four
//     48 KB stages, arming the stage's "full" mbarrier with the byte count;
//   warp 1 (one thread): the MMA issuer.  Per K block it waits for a full
//     stage, issues four tcgen05.mma (M 128, N 256, K 16) into one of two
//     256-column TMEM accumulators and commits them to the stage's "empty"
//     mbarrier; after a tile's last block it commits to the accumulator's
//     "tmem full" mbarrier;
//   warps 2-5: the epilogue.  Each reads its 32-lane quarter of a finished
//     accumulator with tcgen05.ld, adds the bias, applies ReLU or a mask (the
//     backward pass's ReLU derivative), stores bf16 or FP32 rows, and arrives
//     on the accumulator's "tmem empty" mbarrier.
// With two accumulators, the epilogue of one tile overlaps the loads and
// MMAs of the next.
//
// Every wait is bounded: a wait that does not complete within 2 s records an
// error in *err; the CTA then skips the rest of its work and still frees its
// TMEM.
#include <algorithm>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "hedl_internal.h"

namespace hedl {
namespace {

constexpr int UM = 128, UN = 256, UK = 64, STAGES = 4;
constexpr uint32_t ROW = UK * 2;                     // 128-byte rows of a block
constexpr uint32_t A_BYTES = UM * UK * 2;            // 16 KB
constexpr uint32_t B_BYTES = UN * UK * 2;            // 32 KB
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;  // 48 KB
constexpr uint32_t TMEM_COLS = 2 * UN;               // two FP32 accumulators
constexpr int THREADS = 192;                         // producer, MMA issuer, 4 epilogue warps
constexpr size_t UMMA_SMEM = STAGES * STAGE_BYTES + 1024 + 256;

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bit 17,
// M / 16 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UN >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);

// Shared-memory matrix descriptor of a K-major SWIZZLE_128B operand
// (128-byte rows as TMA wrote them): start address / 16 (a K step of 16
// elements advances it by 32 bytes inside the swizzle atom), leading byte
// offset unused (1), stride byte offset (next 8 rows: 1024 B) / 16,
// descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((8u * ROW) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits (one thread) until the barrier's phase of this parity completed, or
// the CTA gave up (*okp cleared elsewhere); false after 2 s or on give-up.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile uint32_t *okp) {
    const uint64_t t0 = now_ns();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255u) == 255u && (!*okp || now_ns() - t0 > 2000000000ull)) return false;
    }
}

__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(ta)
        : "memory");
}

// Fused output layer on 32 columns of one row: the bf16-rounded activations
// (what the unfused path stores and reads back) dotted with both rows of w3.
__device__ __forceinline__ void head32(const UmmaArgs &g, int col, const float (&v)[32], float &a0, float &a1) {
    const uint4 *w0 = reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat16 *>(g.w3) + col);
    const uint4 *w1 = reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat16 *>(g.w3) + g.N + col);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 x = __ldg(w0 + q), y = __ldg(w1 + q);
        const uint32_t xv[4] = {x.x, x.y, x.z, x.w}, yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const __nv_bfloat162 wx = *reinterpret_cast<const __nv_bfloat162 *>(&xv[e]);
            const __nv_bfloat162 wy = *reinterpret_cast<const __nv_bfloat162 *>(&yv[e]);
            const __nv_bfloat162 h = __floats2bfloat162_rn(v[q * 8 + 2 * e], v[q * 8 + 2 * e + 1]);
            const float hl = __low2float(h), hh = __high2float(h);
            a0 += hl * __low2float(wx) + hh * __high2float(wx);
            a1 += hl * __low2float(wy) + hh * __high2float(wy);
        }
    }
}

// Epilogue of 32 columns of one row: bias, ReLU or mask, bf16 or FP32 store
// (and the fused output layer's partial sums).
__device__ __forceinline__ void emit32(const UmmaArgs &g, int row, int col, const uint32_t (&r)[32], float &a0,
                                       float &a1) {
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        float x = __uint_as_float(r[j]);
        if (g.bias) x += g.bias[col + j];
        if (g.relu) x = fmaxf(x, 0.f);
        v[j] = x;
    }
    if (g.mask) {   // keep where the mask (e.g. the forward activation) is positive
        const uint4 *mk =
            reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat16 *>(g.mask) + (size_t)row * g.ldc + col);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 m4 = mk[q];
            const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&mw[e]);
                if (!(__low2float(h) > 0.f)) v[q * 8 + 2 * e] = 0.f;
                if (!(__high2float(h) > 0.f)) v[q * 8 + 2 * e + 1] = 0.f;
            }
        }
    }
    if (g.w3) head32(g, col, v, a0, a1);
    if (!g.store) return;
    if (g.out_bf16) {
        uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(g.C) + (size_t)row * g.ldc + col);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 h = __floats2bfloat162_rn(v[q * 8 + 2 * e], v[q * 8 + 2 * e + 1]);
                w[e] = *reinterpret_cast<const uint32_t *>(&h);
            }
            dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(g.C) + (size_t)row * g.ldc + col);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
}

__global__ void __launch_bounds__(THREADS, 1) umma_kernel(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB, UmmaArgs g) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *tfull = empty + STAGES;    // [2]: accumulator ready for the epilogue
    uint64_t *tempty = tfull + 2;        // [2]: accumulator drained by the epilogue
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile uint32_t *okp = tslot + 1;
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const uint32_t s0 = smem_u32(base);
    const uint32_t full0 = smem_u32(full), empty0 = smem_u32(empty), tfull0 = smem_u32(tfull),
                   tempty0 = smem_u32(tempty);

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8u * i) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8u * i) : "memory");
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull0 + 8u * i) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(tempty0 + 8u * i) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *okp = 1u;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = *tslot;

    const int nk = g.K / UK;
    const int tiles_n = g.N / UN, tiles = ((g.M + UM - 1) / UM) * tiles_n;

    if (warp == 0 && lane == 0) {
        // producer: the running block count u uses stage u % STAGES
        uint32_t u = 0;
        for (int t = blockIdx.x; t < tiles && *okp; t += gridDim.x) {
            const int m0 = (t / tiles_n) * UM, n0 = (t % tiles_n) * UN;
            for (int kb = 0; kb < nk; ++kb, ++u) {
                const uint32_t st = u % STAGES;
                if (u >= STAGES && !mbar_wait(empty0 + 8u * st, ((u - STAGES) / STAGES) & 1u, okp)) {
                    *okp = 0u;
                    break;
                }
                const uint32_t fb = full0 + 8u * st, sa = s0 + st * STAGE_BYTES;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE_BYTES)
                             : "memory");
                tma_2d(sa, &tmA, kb * UK, m0, fb);
                tma_2d(sa + A_BYTES, &tmB, kb * UK, n0, fb);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: the CTA's j-th tile accumulates into buffer j & 1
        uint32_t u = 0, j = 0;
        for (int t = blockIdx.x; t < tiles && *okp; t += gridDim.x, ++j) {
            const uint32_t bf = j & 1u;
            if (j >= 2 && !mbar_wait(tempty0 + 8u * bf, ((j >> 1) - 1u) & 1u, okp)) {
                *okp = 0u;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc_t = taddr + bf * UN;
            bool good = true;
            for (int kb = 0; kb < nk; ++kb, ++u) {
                const uint32_t st = u % STAGES;
                if (!mbar_wait(full0 + 8u * st, (u / STAGES) & 1u, okp)) {
                    *okp = 0u;
                    good = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = s0 + st * STAGE_BYTES;
#pragma unroll
                for (int s = 0; s < UK / 16; ++s) {
                    const uint64_t ad = smem_desc(sa + (uint32_t)s * 32u);
                    const uint64_t bd = smem_desc(sa + A_BYTES + (uint32_t)s * 32u);
                    const uint32_t acc = (kb > 0 || s > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_t),
                        "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 empty0 + 8u * st)
                             : "memory");
            }
            if (!good) break;
            // every MMA issued so far completes before this arrives
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tfull0 + 8u * bf)
                         : "memory");
        }
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, the tile rows of that quarter
        const uint32_t q = warp & 3u;
        uint32_t j = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
            const uint32_t bf = j & 1u;
            uint32_t ok = 1u;
            if (lane == 0) ok = mbar_wait(tfull0 + 8u * bf, (j >> 1) & 1u, okp) ? 1u : 0u;
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
            if (!ok) {
                if (lane == 0) *okp = 0u;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (t / tiles_n) * UM, n0 = (t % tiles_n) * UN;
            const int row = m0 + (int)(q * 32 + lane);
            float a0 = 0.f, a1 = 0.f;   // the fused output layer's partial sums over this tile's columns
            for (int c0 = 0; c0 < UN; c0 += 64) {   // two 32-column loads in flight per wait
                uint32_t ra[32], rb[32];
                const uint32_t ta = taddr + ((q * 32u) << 16) + bf * UN + (uint32_t)c0;
                tmem_ld32(ta, ra);
                tmem_ld32(ta + 32u, rb);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < g.M) {
                    emit32(g, row, n0 + c0, ra, a0, a1);
                    emit32(g, row, n0 + c0 + 32, rb, a0, a1);
                }
            }
            if (g.w3 && row < g.M) {
                atomicAdd(g.y + 2 * (size_t)row, a0);
                atomicAdd(g.y + 2 * (size_t)row + 1, a1);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tempty0 + 8u * bf) : "memory");
        }
    }
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0 && !*okp && g.err) atomicOr(g.err, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}

}  // namespace

bool umma_shape_ok(const UmmaArgs &a) {
    return a.N % UN == 0 && a.K % UK == 0 && a.K > 0 && a.lda % 8 == 0 && a.ldb % 8 == 0 &&
           a.ldc % (a.out_bf16 ? 8 : 4) == 0 && ((uintptr_t)a.A & 15) == 0 && ((uintptr_t)a.B & 15) == 0 &&
           ((uintptr_t)a.C & 15) == 0 && (!a.mask || (a.ldc % 8 == 0 && ((uintptr_t)a.mask & 15) == 0)) &&
           (!a.w3 || (a.y && ((uintptr_t)a.w3 & 15) == 0 && a.N % 8 == 0));
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// Tensor map of a row-major bf16 matrix [rows][ld] (cols used): 64-column x box_rows
// boxes in the 128-byte swizzle, rows past the end read as zeros.
bool make_map(CUtensorMap *m, const void *ptr, int rows, int cols, int ld, int box_rows) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)UK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int umma_gemm(const UmmaArgs &a, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (!umma_shape_ok(a)) return (int)cudaErrorInvalidValue;
    if (a.M <= 0) return 0;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UMMA_SMEM);
        if (e) return (int)e;
        attr = true;
    }
    CUtensorMap ta, tb;
    if (!make_map(&ta, a.A, a.M, a.K, a.lda, UM) || !make_map(&tb, a.B, a.N, a.K, a.ldb, UN))
        return (int)cudaErrorInvalidValue;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) || sms < 1) sms = 1;
    }
    const long tiles = (long)((a.M + UM - 1) / UM) * (a.N / UN);
    umma_kernel<<<(unsigned)std::min<long>(tiles, sms), THREADS, UMMA_SMEM, s>>>(ta, tb, a);
    return (int)cudaGetLastError();
}

}  // namespace hedl
