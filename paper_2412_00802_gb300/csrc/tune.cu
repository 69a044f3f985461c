// Launch-shape autotuner: times candidate tunings of the interpreter on a
// probe batch and keeps the fastest.  Results can be cached in a text file,
// one line per (GPU, KB shape):  <key> warps wpl rounds stage role_block
#include <cuda_runtime.h>

#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "hedl_internal.h"

namespace hedl {
namespace {

bool same_shape(const Tuning &a, const Tuning &b) {
    return a.warps == b.warps && a.wpl == b.wpl && a.rounds == b.rounds && a.stage == b.stage &&
           a.role_block == b.role_block && a.full_occupancy == b.full_occupancy;
}

std::vector<Tuning> candidates(const Tuning &base) {
    std::vector<Tuning> out;
    for (uint32_t stage : {1u, 0u})
        for (uint32_t warps : {8u, 16u, 32u})
            for (uint32_t rounds : {1u, 2u, 4u})
                for (uint32_t blk : {4u, 8u}) {
                    Tuning t = base;
                    t.stage = stage;
                    t.warps = warps;
                    t.wpl = 1;
                    t.rounds = rounds;
                    t.role_block = blk;
                    t.ctas_per_sm = 0;
                    t.full_occupancy = 0;
                    out.push_back(t);
                }
    for (uint32_t warps : {1u, 2u})
        for (uint32_t rounds : {1u, 2u, 4u})
            for (uint32_t blk : {4u, 8u}) {
                Tuning t = base;
                t.stage = 0;
                t.warps = warps;
                t.wpl = 1;
                t.rounds = rounds;
                t.role_block = blk;
                t.ctas_per_sm = 0;
                t.full_occupancy = 0;
                out.push_back(t);
            }
    for (uint32_t rounds : {1u, 2u, 4u})
        for (uint32_t blk : {4u, 8u}) {
            Tuning t = base;
            t.stage = 0;
            t.warps = 8;
            t.wpl = 1;
            t.rounds = rounds;
            t.role_block = blk;
            t.ctas_per_sm = 0;
            t.full_occupancy = 1;
            out.push_back(t);
        }
    for (uint32_t stage : {1u, 0u})
        for (uint32_t warps : {8u, 16u}) {
            Tuning t = base;
            t.stage = stage;
            t.warps = warps;
            t.wpl = 4;
            t.rounds = 1;
            t.role_block = 8;
            t.ctas_per_sm = 0;
            t.full_occupancy = 0;
            out.push_back(t);
        }
    return out;
}

bool fits(const hedl_kb *kb, const Tuning &t) { return stack_smem_bytes(t) + 16 <= kb->smem_optin; }

std::string cache_key(const hedl_kb *kb) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, kb->device);
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
    mix(kb->n);
    mix(kb->n_concepts);
    mix(kb->n_roles);
    mix(kb->n_props);
    for (uint32_t e : kb->role_edges) mix(e);
    if (kb->n_num || kb->n_str) {   // concrete roles (absent: the key of a KB without them is unchanged)
        mix(kb->n_num);
        for (const DevNum &g : kb->num_host) mix(g.n_vals);
        mix(kb->n_str);
        for (const DevStr &g : kb->str_host) mix(g.n_vals);
        mix(kb->n_strings);
        mix(kb->n_patterns);
    }
    for (const char *c = prop.name; *c; ++c) mix((uint8_t)*c);
    mix((uint64_t)prop.multiProcessorCount);
    char buf[64];
    snprintf(buf, sizeof buf, "%016llx", (unsigned long long)h);
    return buf;
}

bool cache_lookup(const char *path, const std::string &key, Tuning *t) {
    std::ifstream f(path);
    std::string line;
    bool found = false;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string k;
        Tuning c = *t;
        if (is >> k >> c.warps >> c.wpl >> c.rounds >> c.stage >> c.role_block >> c.full_occupancy && k == key) {
            *t = c;       // the last matching line wins
            found = true;
        }
    }
    return found;
}

}  // namespace
}  // namespace hedl

using namespace hedl;

extern "C" int hedl_autotune_workspace_size(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H,
                                            size_t *bytes) {
    if (!kb || !bytes) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    const Tuning saved = kb->tuning;
    size_t need = 0;
    for (const Tuning &t : candidates(saved)) {
        if (!fits(kb, t)) continue;
        kb->tuning = t;
        PlanImpl *p = nullptr;
        int e = build_plan(kb, progs, offs, H, 0, &p);
        kb->tuning = saved;
        if (e) return e;
        need = std::max<size_t>(need, p->ws_bytes);
        delete p;
    }
    *bytes = need;
    return HEDL_OK;
}

extern "C" int hedl_autotune(hedl_kb *kb, const uint64_t *progs, const uint32_t *offs, uint32_t H, void *ws,
                             size_t ws_bytes, const char *cache_path, hedl_stream s, hedl_tuning *chosen) {
    if (!kb) return fail(HEDL_ERR_INVALID_ARG, "NULL argument");
    if (kb->plan_only) return fail(HEDL_ERR_INVALID_ARG, "planning-only handle");
    if (!kb->has_examples) return fail(HEDL_ERR_NO_EXAMPLES, "the autotuner scores the probe: set examples first");
    const Tuning saved = kb->tuning;
    Tuning best = saved;
    const std::string key = cache_key(kb);
    bool cached = cache_path && cache_lookup(cache_path, key, &best);
    if (!cached) {
        cudaStream_t st = (cudaStream_t)s;
        uint32_t *counts = nullptr;
        // counts live at the end of ws, past every candidate's plan
        size_t cbytes = 16ull * H;
        size_t need = 0;
        int e = hedl_autotune_workspace_size(kb, progs, offs, H, &need);
        if (e) return e;
        size_t coff = (need + 255) & ~size_t(255);
        if (!ws || ws_bytes < coff + cbytes)
            return fail(HEDL_ERR_WORKSPACE_TOO_SMALL, "autotune workspace of " + std::to_string(ws_bytes) +
                                                          " bytes, " + std::to_string(coff + cbytes) + " needed");
        counts = (uint32_t *)((uint8_t *)ws + coff);
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        float best_ms = 1e30f, saved_ms = -1.f;
        Tuning saved_shape = saved;
        for (const Tuning &t : candidates(saved)) {
            if (!fits(kb, t)) continue;
            kb->tuning = t;
            PlanImpl *p = nullptr;
            e = build_plan(kb, progs, offs, H, HEDL_NO_GRAPH, &p);
            if (e) break;
            e = execute(kb, p, counts, nullptr, ws, coff, s, true);
            float ms = 0;
            for (int rep = 0; rep < 3 && !e; ++rep) {
                cudaEventRecord(a, st);
                e = execute(kb, p, counts, nullptr, ws, coff, s, false);
                cudaEventRecord(b, st);
                cudaError_t ce = cudaEventSynchronize(b);
                if (ce) e = cuda_fail(ce, "autotune timing");
                float m = 0;
                cudaEventElapsedTime(&m, a, b);
                ms += m;
            }
            delete p;
            if (e) break;
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
            if (same_shape(t, saved)) {
                saved_ms = ms;
                saved_shape = t;
            }
        }
        // the current shape stays unless another is at least 2 % faster: timing noise
        // between near-equal shapes must not flip the choice from run to run
        if (!e && saved_ms >= 0.f && saved_ms <= best_ms * 1.02f) best = saved_shape;
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        kb->tuning = saved;
        if (e) return e;
        int se = hedl_sync_status(kb, s);
        if (se) return se;
        if (cache_path) {
            std::ofstream f(cache_path, std::ios::app);
            f << key << ' ' << best.warps << ' ' << best.wpl << ' ' << best.rounds << ' ' << best.stage << ' '
              << best.role_block << ' ' << best.full_occupancy << '\n';
        }
    }
    hedl_tuning ht{best.warps, best.wpl, best.rounds, 0, saved.timeout_ms, best.stage, best.role_block,
                   best.full_occupancy};
    int e = hedl_tuning_set(kb, &ht);
    if (e) return e;
    if (chosen) *chosen = ht;
    return HEDL_OK;
}
