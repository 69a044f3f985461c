// hedl_eval_concept_noalloc: single-program evaluation that allocates no
// memory of its own.
//
// Who needs it: callers that are not allowed to call cudaMalloc (or any other
// device allocator) at the point where they evaluate, for example code
// running under an allocator-free real-time budget, inside a host callback, or
// in a process whose device memory is fully handed to another pool; such a
// caller cannot size and allocate the workspace that hedl_eval_concept wants.
// This variant instead runs the same interpreter kernel on a fixed scratch
// array that the library holds in device memory for the lifetime of the
// process (on every GPU that loads the library).
//
// The scratch is a file-scope __device__ array.  Host code cannot use its name
// as a device address (on the host the name is only a stand-in symbol), so the
// first call on each device, with that device current, looks the address up
// with cudaGetSymbolAddress and remembers it together with the device's
// current context; later calls on that device reuse it while the context is
// the same one.  After cudaDeviceReset (or any teardown that gives the device
// a new primary context) the module is loaded again, possibly at another
// address, so the next call looks the address up again.  Make the first call
// on a device, and the first call after such a reset, before any stream
// capture.
//
// Every call shares the one array: the plan image copied in at each call
// brings its own zeroed counters (the queue head, the per-segment completion
// counts and the coverage accumulators must start at zero), and every slot is
// written before it is read, so nothing is carried over between calls.  Two
// calls whose GPU work overlaps (different streams, or different host
// threads, without ordering between them) race on the array: order them.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "hedl_internal.h"

namespace {

__device__ __align__(256) uint8_t g_scratch[HEDL_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices];
CUcontext g_scratch_ctx[kMaxDevices];   // the context the address belongs to

// cuCtxGetCurrent through the runtime's driver entry point (the library links
// the static runtime only, not libcuda).
using CtxGetCurrent = CUresult (*)(CUcontext *);
CtxGetCurrent ctx_get_current() {
    static const CtxGetCurrent fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (CtxGetCurrent) nullptr;
        return reinterpret_cast<CtxGetCurrent>(p);
    }();
    return fn;
}

// Device address of g_scratch on the current device: looked up once per
// device and context.
int scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return hedl::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return hedl::fail(HEDL_ERR_INVALID_ARG, "device ordinal out of range");
    e = cudaSetDevice(dev);   // makes the device's primary context current on this thread (no allocation)
    if (e) return hedl::cuda_fail(e, "cudaSetDevice");
    CtxGetCurrent get = ctx_get_current();
    if (!get) return hedl::fail(HEDL_ERR_CUDA, "cuCtxGetCurrent is not available from the driver");
    CUcontext ctx = nullptr;
    if (get(&ctx) != CUDA_SUCCESS || !ctx) return hedl::fail(HEDL_ERR_CUDA, "no current CUDA context");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e) return hedl::cuda_fail(e, "cudaGetSymbolAddress of the built-in scratch");
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return HEDL_OK;
}

}  // namespace

extern "C" int hedl_eval_concept_noalloc(hedl_kb *kb, const uint64_t *prog, uint32_t len, uint32_t *out_bits,
                                         hedl_stream s) {
    using namespace hedl;
    if (!kb || !out_bits) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (kb->plan_only) return fail(HEDL_ERR_INVALID_ARG, "planning-only handle");
    void *scratch = nullptr;
    int e = scratch_address(&scratch);
    if (e) return e;
    const uint32_t offs[2] = {0, len};
    const PlanImpl *p = nullptr;
    // direct launches only: building a CUDA graph would create driver objects
    e = cached_plan(kb, prog, offs, 1, HEDL_NO_GRAPH, &p);
    if (e) return e;
    if (p->ws_bytes > (uint64_t)HEDL_NOALLOC_SCRATCH_BYTES)
        return fail(HEDL_ERR_WORKSPACE_TOO_SMALL,
                    "the program needs " + std::to_string(p->ws_bytes) + " bytes of scratch; the built-in scratch of "
                    "hedl_eval_concept_noalloc holds " + std::to_string((uint64_t)HEDL_NOALLOC_SCRATCH_BYTES) +
                    " (use hedl_eval_concept with a larger workspace)");
    return execute(kb, p, nullptr, out_bits, scratch, HEDL_NOALLOC_SCRATCH_BYTES, s, true);
}
