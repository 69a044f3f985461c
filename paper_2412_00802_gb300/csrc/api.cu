// The C ABI (include/hedl.h): argument checks, handle management, plan
// caching, workspace checks, CUDA-graph replay and error reporting.  All
// evaluation work is done by the kernels in exec.cu / plain.cu / kb.cu.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "hedl_internal.h"

namespace hedl {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(int cuda_err, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString((cudaError_t)cuda_err);
    return HEDL_ERR_CUDA;
}

}  // namespace hedl

using namespace hedl;

hedl::KBView hedl_kb::view() const {
    KBView v{};
    v.concepts = concepts;
    v.csr = csr_dev;
    v.num = num_dev;
    v.str = str_dev;
    v.contain = contain_dev;
    v.contain_words = contain_words;
    v.props = props;
    v.prop_stride = prop_stride;
    v.pos = pos;
    v.neg = neg;
    v.status = status_dev;
    v.n = n;
    v.w = w;
    v.wp = wp;
    v.n_pos = n_pos;
    v.n_neg = n_neg;
    return v;
}

namespace {

void drop_cached_plan(hedl_kb *kb) {
    if (kb->cached) {
        hedl_plan_free(kb->cached);
        kb->cached = nullptr;
    }
}

void destroy_graph(PlanImpl *p) {
    if (p->graph_exec) {
        cudaGraphExecDestroy((cudaGraphExec_t)p->graph_exec);
        p->graph_exec = nullptr;
    }
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Host checks of the string concrete roles, the table and the patterns.
int check_str_roles(const hedl_kb_desc *d, bool arrays) {
    if (d->n_str_roles > 65536) return fail(HEDL_ERR_INVALID_ARG, "at most 65536 string roles (16-bit ids)");
    if (d->n_str_roles && !d->str_roles) return fail(HEDL_ERR_INVALID_ARG, "str_roles is NULL");
    for (uint32_t q = 0; q < d->n_str_roles; ++q) {
        const hedl_string_role &g = d->str_roles[q];
        if (g.n_vals >= 0x80000000u) return fail(HEDL_ERR_INVALID_ARG, "a string role has 2^31 or more values");
        if (arrays && (!g.row_ptr || (g.n_vals && !g.ids)))
            return fail(HEDL_ERR_INVALID_ARG, "string role " + std::to_string(q) + ": NULL array");
        if (g.n_vals && d->n_strings == 0)
            return fail(HEDL_ERR_INVALID_ARG, "a string role has values but the string table is empty");
    }
    if (arrays && d->n_strings && (!d->str_off || (d->n_str_chars && !d->str_chars)))
        return fail(HEDL_ERR_INVALID_ARG, "str_off / str_chars is NULL");
    if (arrays && d->n_patterns) {
        if (!d->pat_off || d->pat_off[0] != 0 || (d->pat_off[d->n_patterns] && !d->pat_chars))
            return fail(HEDL_ERR_INVALID_ARG, "pat_off is NULL or does not start at 0, or pat_chars is NULL");
        for (uint32_t k = 0; k < d->n_patterns; ++k)
            if (d->pat_off[k + 1] < d->pat_off[k]) return fail(HEDL_ERR_INVALID_ARG, "pat_off decreases");
    }
    return HEDL_OK;
}

// Sizes (and, for a loadable handle, the device arrays) of the string roles.
void take_str_sizes(hedl_kb *kb, const hedl_kb_desc *d, bool arrays) {
    kb->n_str = d->n_str_roles;
    for (uint32_t q = 0; q < d->n_str_roles; ++q)
        kb->str_host.push_back(DevStr{arrays ? d->str_roles[q].row_ptr : nullptr,
                                      arrays ? d->str_roles[q].ids : nullptr, d->str_roles[q].n_vals, 0});
    kb->n_strings = d->n_strings;
    kb->n_str_chars = d->n_str_chars;
    kb->n_patterns = d->n_patterns;
    kb->contain_words = ((uint64_t)d->n_strings + 31) / 32;
    if (arrays) {
        kb->str_off = d->str_off;
        kb->str_chars = d->str_chars;
    }
}

// Host checks of the numeric concrete roles of a descriptor (arrays only when
// the handle will read them).
int check_num_roles(const hedl_kb_desc *d, bool arrays) {
    if ((uint64_t)d->n_props + d->n_num_roles > 65536)
        return fail(HEDL_ERR_INVALID_ARG, "at most 65536 properties and numeric roles together (16-bit ids)");
    if (d->n_num_roles && !d->num_roles) return fail(HEDL_ERR_INVALID_ARG, "num_roles is NULL");
    for (uint32_t q = 0; q < d->n_num_roles; ++q) {
        const hedl_numeric_role &g = d->num_roles[q];
        if (g.n_vals >= 0x80000000u) return fail(HEDL_ERR_INVALID_ARG, "a numeric role has 2^31 or more values");
        if (arrays && (!g.row_ptr || (g.n_vals && !g.vals)))
            return fail(HEDL_ERR_INVALID_ARG, "numeric role " + std::to_string(q) + ": NULL array");
    }
    return HEDL_OK;
}

}  // namespace

extern "C" {

uint32_t hedl_row_words(uint32_t n_indiv) {
    uint32_t w = (uint32_t)(((uint64_t)n_indiv + 31) / 32);
    return (w + 3) / 4 * 4;
}

const char *hedl_last_error(void) { return g_last_error.c_str(); }

int hedl_kb_load(const hedl_kb_desc *d, unsigned flags, hedl_stream s, hedl_kb **out) {
    if (!out) return fail(HEDL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return fail(HEDL_ERR_INVALID_ARG, "desc is NULL");
    if (d->n_indiv == 0 || d->n_indiv > 0x7FFFFF00u) return fail(HEDL_ERR_INVALID_ARG, "n_indiv must be in [1, 2^31)");
    if (d->n_concepts && !d->concept_bits) return fail(HEDL_ERR_INVALID_ARG, "concept_bits is NULL");
    if (d->n_concepts > 65536 || d->n_roles > 65536 || d->n_props > 65536)
        return fail(HEDL_ERR_INVALID_ARG, "at most 65536 concepts, roles and properties (16-bit ids)");
    if (d->n_roles && (!d->roles || !d->inv_roles)) return fail(HEDL_ERR_INVALID_ARG, "roles / inv_roles is NULL");
    if (d->n_props && (!d->prop_vals || d->prop_stride < d->n_indiv))
        return fail(HEDL_ERR_INVALID_ARG, "prop_vals is NULL or prop_stride < n_indiv");
    if (int e = check_num_roles(d, true)) return e;
    if (int e = check_str_roles(d, true)) return e;
    if (d->concept_bits && !aligned(d->concept_bits, 16))
        return fail(HEDL_ERR_INVALID_ARG, "concept_bits must be 16-byte aligned");
    for (uint32_t r = 0; r < d->n_roles; ++r) {
        const hedl_csr *cs[2] = {&d->roles[r], &d->inv_roles[r]};
        for (const hedl_csr *c : cs) {
            if (!c->row_ptr || (c->n_edges && !c->col))
                return fail(HEDL_ERR_INVALID_ARG, "role " + std::to_string(r) + ": NULL CSR array");
            if (c->n_edges >= 0x80000000u) return fail(HEDL_ERR_INVALID_ARG, "a role has 2^31 or more assertions");
        }
    }
    auto *kb = new hedl_kb();
    kb->n = d->n_indiv;
    kb->w = (d->n_indiv + 31) / 32;
    kb->wp = hedl_row_words(d->n_indiv);
    kb->n_concepts = d->n_concepts;
    kb->n_roles = d->n_roles;
    kb->n_props = d->n_props;
    kb->concepts = d->concept_bits;
    kb->props = d->prop_vals;
    kb->prop_stride = d->prop_stride;
    kb->csr_host.resize(2ull * d->n_roles);
    kb->role_edges.resize(d->n_roles);
    for (uint32_t r = 0; r < d->n_roles; ++r) {
        kb->csr_host[2 * r] = DevCSR{d->roles[r].row_ptr, d->roles[r].col, d->roles[r].n_edges, 0};
        kb->csr_host[2 * r + 1] = DevCSR{d->inv_roles[r].row_ptr, d->inv_roles[r].col, d->inv_roles[r].n_edges, 0};
        kb->role_edges[r] = d->roles[r].n_edges;
    }
    kb->n_num = d->n_num_roles;
    for (uint32_t q = 0; q < d->n_num_roles; ++q)
        kb->num_host.push_back(DevNum{d->num_roles[q].row_ptr, d->num_roles[q].vals, d->num_roles[q].n_vals, 0});
    take_str_sizes(kb, d, true);
    cudaError_t e = cudaGetDevice(&kb->device);
    if (!e) e = cudaDeviceGetAttribute(&kb->n_sms, cudaDevAttrMultiProcessorCount, kb->device);
    int optin = 0;
    if (!e) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, kb->device);
    if (!e) kb->smem_optin = (size_t)optin;
    if (!e) e = cudaMalloc(&kb->status_dev, 8 * sizeof(uint32_t));
    if (!e) e = cudaMemsetAsync(kb->status_dev, 0, 8 * sizeof(uint32_t), (cudaStream_t)s);
    if (!e && d->n_roles) e = cudaMalloc(&kb->csr_dev, sizeof(DevCSR) * kb->csr_host.size());
    if (!e && d->n_roles)
        e = cudaMemcpyAsync(kb->csr_dev, kb->csr_host.data(), sizeof(DevCSR) * kb->csr_host.size(),
                            cudaMemcpyHostToDevice, (cudaStream_t)s);
    if (!e && kb->n_num) e = cudaMalloc(&kb->num_dev, sizeof(DevNum) * kb->n_num);
    if (!e && kb->n_num)
        e = cudaMemcpyAsync(kb->num_dev, kb->num_host.data(), sizeof(DevNum) * kb->n_num, cudaMemcpyHostToDevice,
                            (cudaStream_t)s);
    if (!e && kb->n_str) e = cudaMalloc(&kb->str_dev, sizeof(DevStr) * kb->n_str);
    if (!e && kb->n_str)
        e = cudaMemcpyAsync(kb->str_dev, kb->str_host.data(), sizeof(DevStr) * kb->n_str, cudaMemcpyHostToDevice,
                            (cudaStream_t)s);
    if (!e && kb->n_patterns) {
        const size_t pbytes = d->pat_off[kb->n_patterns];
        e = cudaMalloc(&kb->pat_off_dev, 4ull * (kb->n_patterns + 1));
        if (!e) e = cudaMalloc(&kb->pat_chars_dev, pbytes ? pbytes : 1);
        if (!e)
            e = cudaMemcpyAsync(kb->pat_off_dev, d->pat_off, 4ull * (kb->n_patterns + 1), cudaMemcpyHostToDevice,
                                (cudaStream_t)s);
        if (!e && pbytes)
            e = cudaMemcpyAsync(kb->pat_chars_dev, d->pat_chars, pbytes, cudaMemcpyHostToDevice, (cudaStream_t)s);
        if (!e && kb->contain_words) e = cudaMalloc(&kb->contain_dev, 4ull * kb->contain_words * kb->n_patterns);
    }
    if (!e) e = cudaStreamSynchronize((cudaStream_t)s);
    if (e) {
        int rc = cuda_fail(e, "hedl_kb_load");
        hedl_kb_free(kb);
        return rc;
    }
    if (!(flags & HEDL_KB_NO_VALIDATE)) {
        std::string why;
        int ve = kb_validate_device(kb, s, &why);
        if (ve) {
            int rc = cuda_fail(ve, "hedl_kb_load validation");
            hedl_kb_free(kb);
            return rc;
        }
        if (!why.empty()) {
            hedl_kb_free(kb);
            return fail(HEDL_ERR_BAD_KB, why);
        }
    }
    if (kb->n_patterns) {   // which table strings contain which pattern (the table is valid here)
        int ce = contain_bitmap_device(kb, s);
        if (ce) {
            int rc = cuda_fail(ce, "hedl_kb_load pattern bitmap");
            hedl_kb_free(kb);
            return rc;
        }
    }
    *out = kb;
    return HEDL_OK;
}

int hedl_kb_plan_only(const hedl_kb_desc *d, hedl_kb **out) {
    if (!out) return fail(HEDL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!d) return fail(HEDL_ERR_INVALID_ARG, "desc is NULL");
    if (d->n_indiv == 0 || d->n_indiv > 0x7FFFFF00u) return fail(HEDL_ERR_INVALID_ARG, "n_indiv must be in [1, 2^31)");
    if (d->n_concepts > 65536 || d->n_roles > 65536 || d->n_props > 65536)
        return fail(HEDL_ERR_INVALID_ARG, "at most 65536 concepts, roles and properties (16-bit ids)");
    if (d->n_roles && (!d->roles || !d->inv_roles)) return fail(HEDL_ERR_INVALID_ARG, "roles / inv_roles is NULL");
    if (int e = check_num_roles(d, false)) return e;
    if (int e = check_str_roles(d, false)) return e;
    auto *kb = new hedl_kb();
    kb->plan_only = true;
    kb->n = d->n_indiv;
    kb->w = (d->n_indiv + 31) / 32;
    kb->wp = hedl_row_words(d->n_indiv);
    kb->n_concepts = d->n_concepts;
    kb->n_roles = d->n_roles;
    kb->n_props = d->n_props;
    kb->n_sms = PLAN_ONLY_SMS;
    kb->csr_host.resize(2ull * d->n_roles);
    kb->role_edges.resize(d->n_roles);
    for (uint32_t r = 0; r < d->n_roles; ++r) {
        kb->csr_host[2 * r] = DevCSR{nullptr, nullptr, d->roles[r].n_edges, 0};
        kb->csr_host[2 * r + 1] = DevCSR{nullptr, nullptr, d->inv_roles[r].n_edges, 0};
        kb->role_edges[r] = d->roles[r].n_edges;
    }
    kb->n_num = d->n_num_roles;
    for (uint32_t q = 0; q < d->n_num_roles; ++q) kb->num_host.push_back(DevNum{nullptr, nullptr, d->num_roles[q].n_vals, 0});
    take_str_sizes(kb, d, false);
    *out = kb;
    return HEDL_OK;
}

void hedl_kb_free(hedl_kb *kb) {
    if (!kb) return;
    if (kb->plan_only) {
        drop_cached_plan(kb);
        delete kb;
        return;
    }
    cudaDeviceSynchronize();
    drop_cached_plan(kb);
    if (kb->capture_stream) cudaStreamDestroy((cudaStream_t)kb->capture_stream);
    if (kb->csr_dev) cudaFree(kb->csr_dev);
    if (kb->num_dev) cudaFree(kb->num_dev);
    if (kb->str_dev) cudaFree(kb->str_dev);
    if (kb->pat_off_dev) cudaFree(kb->pat_off_dev);
    if (kb->pat_chars_dev) cudaFree(kb->pat_chars_dev);
    if (kb->contain_dev) cudaFree(kb->contain_dev);
    if (kb->status_dev) cudaFree(kb->status_dev);
    delete kb;
}

int hedl_examples_set(hedl_kb *kb, const uint32_t *pos_bits, const uint32_t *neg_bits, hedl_stream s) {
    if (!kb || !pos_bits || !neg_bits) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (kb->plan_only) return fail(HEDL_ERR_INVALID_ARG, "planning-only handle");
    if (!aligned(pos_bits, 16) || !aligned(neg_bits, 16))
        return fail(HEDL_ERR_INVALID_ARG, "example bitsets must be 16-byte aligned");
    kb->pos = pos_bits;
    kb->neg = neg_bits;
    uint32_t np = 0, nn = 0;
    int e = examples_count_device(kb, s, &np, &nn);
    if (e < 0) {
        kb->pos = kb->neg = nullptr;
        kb->has_examples = false;
        return fail(HEDL_ERR_INVALID_ARG, "an example bitset has bits set beyond n or in its padding words");
    }
    if (e) {
        kb->pos = kb->neg = nullptr;
        kb->has_examples = false;
        return cuda_fail(e, "hedl_examples_set");
    }
    kb->n_pos = np;
    kb->n_neg = nn;
    kb->has_examples = true;
    return HEDL_OK;
}

int hedl_examples_counts(const hedl_kb *kb, uint32_t *n_pos, uint32_t *n_neg) {
    if (!kb || !n_pos || !n_neg) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (!kb->has_examples) return fail(HEDL_ERR_NO_EXAMPLES, "no examples set");
    *n_pos = kb->n_pos;
    *n_neg = kb->n_neg;
    return HEDL_OK;
}

int hedl_validate(const hedl_kb *kb, const uint64_t *prog, uint32_t len) {
    if (!kb || (len && !prog)) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    std::string why;
    int e = validate_program(kb, prog, len, &why);
    if (e) return fail(e, why);
    return HEDL_OK;
}

int hedl_plan_batch(const hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, unsigned flags,
                    hedl_plan **out) {
    if (!out) return fail(HEDL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!kb || !offs || (H && offs[H] && !progs)) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    PlanImpl *impl = nullptr;
    int e = build_plan(kb, progs, offs, H, flags, &impl);
    if (e) return e;
    auto *p = new hedl_plan();
    p->impl = impl;
    *out = p;
    return HEDL_OK;
}

int hedl_plan_info_get(const hedl_plan *p, hedl_plan_info *info) {
    if (!p || !info) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    *info = p->impl->info;
    return HEDL_OK;
}

int hedl_plan_image(const hedl_plan *p, void *out, size_t cap, size_t *bytes) {
    if (!p || !bytes) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (p->impl->dev_image) {   // a device-built plan
        *bytes = p->impl->image_bytes;
        if (!out || cap < *bytes)
            return fail(HEDL_ERR_INVALID_ARG, "image of " + std::to_string(*bytes) + " bytes, buffer of " +
                                                  std::to_string(cap));
        cudaError_t e = cudaMemcpy(out, p->impl->dev_image, *bytes, cudaMemcpyDeviceToHost);
        return e ? cuda_fail(e, "plan image copy") : HEDL_OK;
    }
    const std::vector<uint8_t> &img = p->impl->image;
    *bytes = img.size();
    if (img.empty()) return HEDL_OK;
    if (!out || cap < img.size())
        return fail(HEDL_ERR_INVALID_ARG, "image of " + std::to_string(img.size()) + " bytes, buffer of " +
                                              std::to_string(cap));
    memcpy(out, img.data(), img.size());
    return HEDL_OK;
}

void hedl_plan_free(hedl_plan *p) {
    if (!p) return;
    if (p->impl) {
        destroy_graph(p->impl);
        if (p->impl->dev_image) cudaFree(p->impl->dev_image);
        delete p->impl;
    }
    delete p;
}

}  // extern "C"

int execute(hedl_kb *kb, const PlanImpl *pc, uint32_t *counts, uint32_t *out_bits, void *ws, size_t ws_bytes,
                   hedl_stream s, bool upload) {
    PlanImpl *p = const_cast<PlanImpl *>(pc);
    if (kb->plan_only) return fail(HEDL_ERR_INVALID_ARG, "planning-only handle: nothing can be launched");
    if (!counts && !out_bits) return fail(HEDL_ERR_INVALID_ARG, "counts and out_bits are both NULL");
    if (counts && !kb->has_examples) return fail(HEDL_ERR_NO_EXAMPLES, "scoring needs hedl_examples_set first");
    if (!ws || ws_bytes < p->ws_bytes)
        return fail(HEDL_ERR_WORKSPACE_TOO_SMALL,
                    "workspace of " + std::to_string(ws_bytes) + " bytes, " + std::to_string(p->ws_bytes) + " needed");
    if (!aligned(ws, 256)) return fail(HEDL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if ((counts && !aligned(counts, 16)) || (out_bits && !aligned(out_bits, 16)))
        return fail(HEDL_ERR_INVALID_ARG, "counts and out_bits must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)s;
    if (p->flags & HEDL_PLAIN) {
        int e = launch_plain(kb, p, counts, out_bits, ws, st);
        return e ? cuda_fail(e, "plain launch") : HEDL_OK;
    }
    if (p->bps == 0) {  // launch shape, resolved outside any stream capture
        int bps = 0;
        int oe = exec_occupancy(kb, p->tuning, p->n_rgroups > 0, &bps);
        if (oe) return cuda_fail(oe, "occupancy query");
        if (bps < 1) return fail(HEDL_ERR_CUDA, "the interpreter kernel does not fit on an SM");
        p->bps = bps;
    }
    cudaError_t e;
    if (upload && p->dev_image) {
        // a device-built plan: its image is copied within the device
        e = cudaMemcpyAsync(ws, p->dev_image, p->image_bytes, cudaMemcpyDeviceToDevice, st);
        if (e) return cuda_fail(e, "plan copy");
    } else if (upload) {
        // pageable source: the copy is complete (staged) when the call returns,
        // so the host image may be reused at once
        e = cudaMemcpyAsync(ws, p->image.data(), p->image_bytes, cudaMemcpyHostToDevice, st);
        if (e) return cuda_fail(e, "plan upload");
    } else {
        e = cudaMemsetAsync((uint8_t *)ws + p->ctr_off, 0, p->ctr_bytes, st);
        if (e) return cuda_fail(e, "counter reset");
    }
    const bool use_graph = !(p->flags & (HEDL_NO_GRAPH | HEDL_LEVELS)) && p->runs++ > 0;
    if (!use_graph) {
        int le = launch_exec(kb, p, counts, out_bits, ws, st);
        return le ? cuda_fail(le, "exec launch") : HEDL_OK;
    }
    if (!p->graph_exec || p->graph_ws != ws || p->graph_counts != counts || p->graph_out != out_bits) {
        destroy_graph(p);
        // captured on the handle's own stream (the legacy default stream
        // cannot be captured), launched on the caller's
        if (!kb->capture_stream) {
            cudaStream_t cs;
            e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e) return cuda_fail(e, "capture stream");
            kb->capture_stream = cs;
        }
        cudaStream_t cs = (cudaStream_t)kb->capture_stream;
        cudaGraph_t g;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e) return cuda_fail(e, "graph capture");
        int le = launch_exec(kb, p, counts, out_bits, ws, cs);
        e = cudaStreamEndCapture(cs, &g);
        if (le) return cuda_fail(le, "exec launch (capture)");
        if (e) return cuda_fail(e, "graph capture end");
        cudaGraphExec_t ge;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e) return cuda_fail(e, "graph instantiate");
        p->graph_exec = ge;
        p->graph_ws = ws;
        p->graph_counts = counts;
        p->graph_out = out_bits;
    }
    e = cudaGraphLaunch((cudaGraphExec_t)p->graph_exec, st);
    return e ? cuda_fail(e, "graph launch") : HEDL_OK;
}

extern "C" {


int hedl_plan_execute(hedl_kb *kb, const hedl_plan *p, uint32_t *counts, uint32_t *out_bits, void *ws,
                      size_t ws_bytes, hedl_stream s) {
    if (!kb || !p) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    return execute(kb, p->impl, counts, out_bits, ws, ws_bytes, s, true);
}

int hedl_plan_replay(hedl_kb *kb, const hedl_plan *p, uint32_t *counts, uint32_t *out_bits, void *ws,
                     size_t ws_bytes, hedl_stream s) {
    if (!kb || !p) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    return execute(kb, p->impl, counts, out_bits, ws, ws_bytes, s, false);
}

}  // extern "C"

int cached_plan(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, unsigned flags,
                       const PlanImpl **out) {
    if (!offs || (H && offs[H] && !progs)) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (H == 0) return fail(HEDL_ERR_INVALID_ARG, "empty batch (H = 0)");
    uint64_t h = hash_programs(progs, offs, H);
    if (kb->cached && kb->cached_hash == h && kb->cached_flags == flags) {
        // the hash only selects a candidate: the programs themselves must be the cached ones
        const PlanImpl *c = kb->cached->impl;
        if (c->info.n_hyps == H && c->info.total_insns == offs[H] && kb->cached_offs.size() == (size_t)H + 1 &&
            memcmp(kb->cached_offs.data(), offs, 4ull * (H + 1)) == 0 &&
            (offs[H] == 0 || memcmp(kb->cached_progs.data(), progs, 8ull * offs[H]) == 0)) {
            *out = c;
            return HEDL_OK;
        }
    }
    hedl_plan *np = nullptr;
    int e = hedl_plan_batch(kb, progs, offs, H, flags, &np);
    if (e) return e;
    drop_cached_plan(kb);
    kb->cached = np;
    kb->cached_hash = h;
    kb->cached_flags = flags;
    kb->cached_offs.assign(offs, offs + H + 1);
    kb->cached_progs.assign(progs, progs + offs[H]);
    *out = np->impl;
    return HEDL_OK;
}

extern "C" {


int hedl_workspace_size(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, unsigned flags,
                        size_t *bytes) {
    if (!kb || !bytes) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    const PlanImpl *p = nullptr;
    int e = cached_plan(kb, progs, offs, H, flags, &p);
    if (e) return e;
    *bytes = p->ws_bytes;
    return HEDL_OK;
}

int hedl_score_batch(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, uint32_t *counts,
                     void *ws, size_t ws_bytes, unsigned flags, hedl_stream s) {
    if (!kb || !counts) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    const PlanImpl *p = nullptr;
    int e = cached_plan(kb, progs, offs, H, flags, &p);
    if (e) return e;
    return execute(kb, p, counts, nullptr, ws, ws_bytes, s, true);
}

int hedl_eval_concept(hedl_kb *kb, const uint64_t *prog, uint32_t len, uint32_t *out_bits, void *ws,
                      size_t ws_bytes, unsigned flags, hedl_stream s) {
    if (!kb || !out_bits) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    const uint32_t offs[2] = {0, len};
    const PlanImpl *p = nullptr;
    int e = cached_plan(kb, prog, offs, 1, flags, &p);
    if (e) return e;
    return execute(kb, p, nullptr, out_bits, ws, ws_bytes, s, true);
}

int hedl_sync_status(hedl_kb *kb, hedl_stream s) {
    if (!kb) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (kb->plan_only) return fail(HEDL_ERR_INVALID_ARG, "planning-only handle");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)s);
    if (e) return cuda_fail(e, "stream synchronize");
    uint32_t st = 0;
    e = cudaMemcpy(&st, kb->status_dev, 4, cudaMemcpyDeviceToHost);
    if (e) return cuda_fail(e, "status read");
    if (st) {
        e = cudaMemset(kb->status_dev, 0, 4);
        if (e) return cuda_fail(e, "status reset");
    }
    if (st & ST_TIMEOUT) return fail(HEDL_ERR_TIMEOUT, "a device-side dependency wait gave up (timeout)");
    return HEDL_OK;
}

int hedl_tuning_get(const hedl_kb *kb, hedl_tuning *t) {
    if (!kb || !t) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    t->warps_per_cta = kb->tuning.warps;
    t->words_per_lane = kb->tuning.wpl;
    t->rounds = kb->tuning.rounds;
    t->ctas_per_sm = kb->tuning.ctas_per_sm;
    t->wait_timeout_ms = kb->tuning.timeout_ms;
    t->stage_fillers = kb->tuning.stage;
    t->role_block = kb->tuning.role_block;
    t->full_occupancy = kb->tuning.full_occupancy;
    return HEDL_OK;
}

int hedl_tuning_set(hedl_kb *kb, const hedl_tuning *t) {
    if (!kb || !t) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (!(t->warps_per_cta == 1 || t->warps_per_cta == 2 || t->warps_per_cta == 4 || t->warps_per_cta == 8 ||
          t->warps_per_cta == 16 || t->warps_per_cta == 32))
        return fail(HEDL_ERR_INVALID_ARG, "warps_per_cta must be 1, 2, 4, 8, 16 or 32");
    if (t->warps_per_cta < 4 && t->words_per_lane != 1)
        return fail(HEDL_ERR_INVALID_ARG, "warps_per_cta 1 and 2 take words_per_lane 1");
    if (t->stage_fillers > 1) return fail(HEDL_ERR_INVALID_ARG, "stage_fillers must be 0 or 1");
    if (!(t->role_block == 4 || t->role_block == 8)) return fail(HEDL_ERR_INVALID_ARG, "role_block must be 4 or 8");
    if (t->full_occupancy > 1) return fail(HEDL_ERR_INVALID_ARG, "full_occupancy must be 0 or 1");
    if (t->words_per_lane == 4 && t->warps_per_cta == 32)
        return fail(HEDL_ERR_INVALID_ARG, "words_per_lane 4 supports at most 16 warps per CTA");
    {
        Tuning probe = kb->tuning;
        probe.warps = t->warps_per_cta;
        probe.wpl = t->words_per_lane;
        if (stack_smem_bytes(probe) + 16 > kb->smem_optin)
            return fail(HEDL_ERR_INVALID_ARG, "warps_per_cta x words_per_lane: the interpreter's stack (" +
                                                  std::to_string(stack_smem_bytes(probe)) +
                                                  " bytes) does not fit in a CTA's shared memory");
    }
    if (!(t->words_per_lane == 1 || t->words_per_lane == 4))
        return fail(HEDL_ERR_INVALID_ARG, "words_per_lane must be 1 or 4");
    if (t->rounds < 1 || t->rounds > 64) return fail(HEDL_ERR_INVALID_ARG, "rounds must be in 1..64");
    if (t->wait_timeout_ms < 1 || t->wait_timeout_ms > 60000)
        return fail(HEDL_ERR_INVALID_ARG, "wait_timeout_ms must be in 1..60000");
    kb->tuning.warps = t->warps_per_cta;
    kb->tuning.wpl = t->words_per_lane;
    kb->tuning.rounds = t->rounds;
    kb->tuning.ctas_per_sm = t->ctas_per_sm;
    kb->tuning.timeout_ms = t->wait_timeout_ms;
    kb->tuning.stage = t->stage_fillers;
    kb->tuning.role_block = t->role_block;
    kb->tuning.full_occupancy = t->full_occupancy;
    drop_cached_plan(kb);
    return HEDL_OK;
}

}  // extern "C"
