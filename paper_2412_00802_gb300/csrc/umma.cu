// Dense layer GEMM of the surrogate on the 5th-generation tensor cores:
// C[M][N] = act(A[M][K] . B[N][K]^T + bias), A and B bf16 and K-major (rows
// of K contiguous elements), FP32 accumulation in tensor memory (TMEM).
//
// One CTA of 4 warps computes a 256 x 256 tile.  K runs in blocks of 32: the
// CTA's threads copy a block of A (256 x 32) and B (256 x 32) into shared
// memory with 16-byte async copies, laid out as 8-row x 16-byte core
// matrices (no swizzle), three blocks ahead in a ring of four stages; one
// thread issues four tcgen05.mma (M 128, N 256, K 16 each: two K steps times
// the two 128-row halves of A, which share the B block) per block and
// commits them to the stage's mbarrier, which frees the stage for reuse.  The
// two 128 x 256 FP32 accumulators fill the SM's 512 TMEM columns (one CTA
// per SM); the epilogue reads them back with tcgen05.ld (each warp its 32
// rows of each half), adds the bias, applies ReLU or a mask (the backward
// pass's ReLU derivative) and stores bf16 or FP32 rows.
//
// Every wait is bounded: if a stage's MMAs do not complete within 2 s, the
// CTA records an error in *err, skips the rest of its work and still frees
// its TMEM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "hedl_internal.h"

namespace hedl {
namespace {

constexpr int UM = 256, UN = 256, UK = 32, STAGES = 4;   // two 128-row MMA halves per tile
constexpr uint32_t KCH = UK / 8;                     // 16-byte K chunks per row and block
constexpr uint32_t SBO = KCH * 128;                  // bytes between 8-row groups of a stage
constexpr uint32_t A_BYTES = UM * UK * 2;            // 16 KB
constexpr uint32_t B_BYTES = UN * UK * 2;            // 16 KB
constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;  // 32 KB
constexpr uint32_t TMEM_COLS = 2 * UN;               // FP32 accumulators of the two halves
constexpr size_t UMMA_SMEM = STAGES * STAGE_BYTES + 1024 + 128;

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at bit 17,
// M / 16 at bit 24.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UN >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);

// Shared-memory matrix descriptor of a K-major operand without swizzle:
// start address / 16, leading byte offset (next 8 K-elements: 128 B) / 16,
// stride byte offset (next 8 rows: SBO) / 16, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

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

// Waits (one thread) until the barrier's phase of this parity completed; false after 2 s.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = now_ns();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255u) == 255u && now_ns() - t0 > 2000000000ull) return false;
    }
}

// Stage one K block: A rows m0.. (zero past M), B rows n0.., 16 bytes a thread per copy.
__device__ __forceinline__ void load_stage(const UmmaArgs &g, uint32_t sA, uint32_t sB, int m0, int n0, int k0) {
    for (int c = threadIdx.x; c < UM * (int)KCH; c += blockDim.x) {
        const int r = c / (int)KCH, kc = c % (int)KCH;
        const bool ok = m0 + r < g.M;
        const __nv_bfloat16 *src =
            reinterpret_cast<const __nv_bfloat16 *>(g.A) + (size_t)(ok ? m0 + r : 0) * g.lda + k0 + kc * 8;
        cp16(sA + (uint32_t)((r >> 3) * SBO + kc * 128 + (r & 7) * 16), src, ok);
    }
    for (int c = threadIdx.x; c < UN * (int)KCH; c += blockDim.x) {
        const int r = c / (int)KCH, kc = c % (int)KCH;
        const __nv_bfloat16 *src = reinterpret_cast<const __nv_bfloat16 *>(g.B) + (size_t)(n0 + r) * g.ldb + k0 + kc * 8;
        cp16(sB + (uint32_t)((r >> 3) * SBO + kc * 128 + (r & 7) * 16), src, true);
    }
}

__global__ void __launch_bounds__(128) umma_kernel(UmmaArgs g) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + STAGES * STAGE_BYTES);     // one per stage
    uint32_t *tslot = reinterpret_cast<uint32_t *>(base + STAGES * STAGE_BYTES + 64);
    uint32_t *okp = reinterpret_cast<uint32_t *>(base + STAGES * STAGE_BYTES + 80);
    const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
    const int n0 = blockIdx.x * UN, m0 = blockIdx.y * UM;
    const uint32_t s0 = smem_u32(base), bar0 = smem_u32(bar);

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * i) : "memory");
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

    // Block kb lives in stage kb % STAGES and its MMAs commit to that stage's
    // barrier (the stage's (kb / STAGES)-th phase).  Copies run STAGES - 1
    // blocks ahead; one async-copy group is committed per block (empty past K).
    const int nk = g.K / UK;
    for (int i = 0; i < STAGES - 1; ++i) {
        if (i < nk) load_stage(g, s0 + i * STAGE_BYTES, s0 + i * STAGE_BYTES + A_BYTES, m0, n0, i * UK);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int kb = 0; kb < nk; ++kb) {
        const uint32_t st = s0 + (uint32_t)(kb % STAGES) * STAGE_BYTES;
        asm volatile("cp.async.wait_group %0;" ::"n"(STAGES - 2) : "memory");
        // make this thread's copies visible to the tensor cores' (async) proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < UK / 16; ++s) {
                const uint64_t bd = smem_desc(st + A_BYTES + (uint32_t)s * 256u);
                const uint32_t acc = (kb > 0 || s > 0) ? 1u : 0u;
#pragma unroll
                for (int h = 0; h < 2; ++h) {   // rows 128h.. of the tile into accumulator columns 256h..
                    const uint64_t ad = smem_desc(st + (uint32_t)h * (16u * SBO) + (uint32_t)s * 256u);
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                            taddr + (uint32_t)h * UN),
                        "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                        : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar0 + 8u * (uint32_t)(kb % STAGES))
                         : "memory");
        }
        // refill the stage block kb-1 used with block kb + STAGES - 1, once its MMAs are done
        const int nx = kb + STAGES - 1;
        if (nx < nk) {
            if (kb >= 1 && threadIdx.x == 0 &&
                !mbar_wait(bar0 + 8u * (uint32_t)((kb - 1) % STAGES), (uint32_t)((kb - 1) / STAGES) & 1u))
                *okp = 0u;
            __syncthreads();
            if (!*okp) break;
            const uint32_t sx = s0 + (uint32_t)(nx % STAGES) * STAGE_BYTES;
            load_stage(g, sx, sx + A_BYTES, m0, n0, nx * UK);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (threadIdx.x == 0 && *okp &&
        !mbar_wait(bar0 + 8u * (uint32_t)((nk - 1) % STAGES), (uint32_t)((nk - 1) / STAGES) & 1u))
        *okp = 0u;
    __syncthreads();
    const bool ok = *okp != 0u;
    if (!ok && threadIdx.x == 0 && g.err) atomicOr(g.err, 1u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    for (int h = 0; ok && h < 2; ++h) {
        const int row = m0 + h * 128 + (int)(warp * 32 + lane);
        for (int c0 = 0; c0 < UN; c0 += 32) {
            uint32_t r[32];
            const uint32_t ta = taddr + ((warp * 32u) << 16) + (uint32_t)(h * UN + c0);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(ta)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < g.M) {
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float x = __uint_as_float(r[j]);
                    if (g.bias) x += g.bias[n0 + c0 + j];
                    if (g.relu) x = fmaxf(x, 0.f);
                    v[j] = x;
                }
                if (g.mask) {   // keep where the mask (e.g. the forward activation) is positive
                    const uint4 *mk = reinterpret_cast<const uint4 *>(reinterpret_cast<const __nv_bfloat16 *>(g.mask) +
                                                                      (size_t)row * g.ldc + n0 + c0);
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
                if (g.out_bf16) {
                    uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(g.C) +
                                                           (size_t)row * g.ldc + n0 + c0);
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
                    float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(g.C) + (size_t)row * g.ldc +
                                                             n0 + c0);
#pragma unroll
                    for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}

}  // namespace

bool umma_shape_ok(const UmmaArgs &a) {
    return a.N % UN == 0 && a.K % UK == 0 && a.K > 0 && a.lda % 8 == 0 && a.ldb % 8 == 0 &&
           a.ldc % (a.out_bf16 ? 8 : 4) == 0 && ((uintptr_t)a.A & 15) == 0 && ((uintptr_t)a.B & 15) == 0 &&
           ((uintptr_t)a.C & 15) == 0 && (!a.mask || (a.ldc % 8 == 0 && ((uintptr_t)a.mask & 15) == 0));
}

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
    dim3 grid((unsigned)(a.N / UN), (unsigned)((a.M + UM - 1) / UM));
    umma_kernel<<<grid, 128, UMMA_SMEM, s>>>(a);
    return (int)cudaGetLastError();
}

}  // namespace hedl
