// Batch groups: any number of lattices of uneven sizes in one CUDA graph.
//
// A batch keeps every member's tensors in its own arena at once, so a set of
// lattices whose summed footprint exceeds the device is split into passes,
// in member order, each pass as large as the pass budget allows.  The passes
// run one after another, so they share one arena (the largest pass's); each
// pass keeps only its small regions (inputs, rescaling slots, dot partials,
// results, task tables) to itself.  The launches of all passes are captured,
// in order, into one CUDA graph on the group's stream: a run of the whole set
// is one graph launch.  A member's program, tiles and reductions depend only
// on its shape, so it gives the same bits in a group as alone.
#include <algorithm>
#include <cstring>
#include <memory>

#include "runtime.h"

namespace tn {
void fill_uniform(uint64_t seed, double* out, size_t n);
}

using namespace tn;

struct tn_batch_group {
    tn_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    int n = 0;
    std::vector<tn_batch*> passes;
    std::vector<std::vector<int>> members;   // member indices of each pass
    char* arena = nullptr;
    size_t arena_bytes = 0;
    cudaGraphExec_t gexec = nullptr;
    std::vector<size_t> in_off, in_elems;    // per member, in the concatenated inputs
    std::vector<size_t> res_off, res_elems;  // per member, in the concatenated results
    size_t nin = 0, nres = 0;
};

namespace {

constexpr uint64_t kGammaG = 0x9E3779B97F4A7C15ull;

uint64_t mix64g(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void group_free(tn_batch_group* g) {
    if (!g) return;
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    for (tn_batch* b : g->passes) batch_destroy(b);
    if (g->arena) {
        cudaFree(g->arena);
        g->ctx->used -= g->arena_bytes;
    }
    delete g;
}

}  // namespace

extern "C" {

tn_status tn_batch_group_create(tn_ctx* ctx, int n, const int* L, const int* W, const int* D, tn_precision prec,
                                tn_schedule sched, tn_work work, size_t pass_budget, tn_batch_group** out) {
    try {
        if (!ctx || !out || n <= 0 || !L || !W || !D || pass_budget == 0) return TN_ERR_INVALID;
        *out = nullptr;
        if (ctx->device < 0) { set_error("context has no device"); return TN_ERR_NO_DEVICE; }
        // each member's footprint alone, for the split into passes; an energy
        // whose cached chain states exceed the pass budget takes the recompute
        // form (the same values, fewer bytes)
        std::vector<size_t> fp(n);
        std::vector<int> kn(n, -1);
        for (int k = 0; k < n; ++k) {
            tn_batch* probe = nullptr;
            tn_status st = batch_create(ctx, 1, &L[k], &W[k], &D[k], prec, sched, work, false, &probe, &fp[k]);
            if (probe) delete probe;
            if (st != TN_OK) return st;
            const int code = tuned_knobs(L[k], W[k], D[k], prec, work).code();
            if (fp[k] > pass_budget && work != TN_WORK_NORM && !(code & kRecomputeKnob)) {
                BatchOpts o;
                o.knobs = code | kRecomputeKnob;
                size_t f2 = 0;
                probe = nullptr;
                st = batch_create(ctx, 1, &L[k], &W[k], &D[k], prec, sched, work, false, &probe, &f2, &o);
                if (probe) delete probe;
                if (st != TN_OK) return st;
                if (f2 <= pass_budget) { fp[k] = f2; kn[k] = o.knobs; }
            }
            if (fp[k] > pass_budget) {
                set_error("member " + std::to_string(k) + " alone needs " + std::to_string(fp[k]) +
                          " B, more than the pass budget");
                return TN_ERR_OVER_BUDGET;
            }
        }
        // freed with everything it holds on every early return or exception
        std::unique_ptr<tn_batch_group, void (*)(tn_batch_group*)> owner(new tn_batch_group(), group_free);
        tn_batch_group* g = owner.get();
        g->ctx = ctx;
        g->stream = ctx->stream;
        g->n = n;
        std::vector<int> cur;
        size_t used = 0;
        for (int k = 0; k < n; ++k) {
            if (!cur.empty() && used + fp[k] > pass_budget) {
                g->members.push_back(cur);
                cur.clear();
                used = 0;
            }
            cur.push_back(k);
            used += fp[k];
        }
        g->members.push_back(cur);
        // the shared arena: the largest pass's
        BatchOpts sizing;
        sizing.arena_external = true;
        for (const auto& mem : g->members) {
            std::vector<int> l, w, d;
            sizing.member_knobs.clear();
            for (int k : mem) {
                l.push_back(L[k]); w.push_back(W[k]); d.push_back(D[k]);
                sizing.member_knobs.push_back(kn[k]);
            }
            tn_batch* probe = nullptr;
            const tn_status st = batch_create(ctx, (int)mem.size(), l.data(), w.data(), d.data(), prec, sched, work,
                                              false, &probe, nullptr, &sizing);
            if (st != TN_OK) { if (probe) delete probe; return st; }
            g->arena_bytes = std::max(g->arena_bytes, probe->arena_bytes);
            delete probe;
        }
        g->arena_bytes = std::max<size_t>(g->arena_bytes, 256);
        size_t cur_used = ctx->used.load();
        do {
            if (cur_used + g->arena_bytes > ctx->budget) {
                g->arena_bytes = 0;
                set_error("the shared arena exceeds the remaining budget");
                return TN_ERR_OVER_BUDGET;
            }
        } while (!ctx->used.compare_exchange_weak(cur_used, cur_used + g->arena_bytes));
        cudaSetDevice(ctx->device);
        cudaError_t e = cudaMalloc(&g->arena, g->arena_bytes);
        if (e != cudaSuccess) {
            ctx->used -= g->arena_bytes;
            g->arena = nullptr;
            g->arena_bytes = 0;
            return cuda_status(e, "shared arena");
        }
        BatchOpts opts;
        opts.arena_external = true;
        opts.ext_arena = g->arena;
        opts.ext_arena_bytes = g->arena_bytes;
        opts.use_graph = false;
        g->in_off.assign(n, 0); g->in_elems.assign(n, 0);
        g->res_off.assign(n, 0); g->res_elems.assign(n, 0);
        for (const auto& mem : g->members) {
            std::vector<int> l, w, d;
            opts.member_knobs.clear();
            for (int k : mem) {
                l.push_back(L[k]); w.push_back(W[k]); d.push_back(D[k]);
                opts.member_knobs.push_back(kn[k]);
            }
            tn_batch* b = nullptr;
            const tn_status st = batch_create(ctx, (int)mem.size(), l.data(), w.data(), d.data(), prec, sched, work,
                                              true, &b, nullptr, &opts);
            if (st != TN_OK) return st;
            g->passes.push_back(b);
        }
        // member order in the concatenated inputs and results
        for (size_t pi = 0; pi < g->passes.size(); ++pi)
            for (size_t j = 0; j < g->members[pi].size(); ++j) {
                const int k = g->members[pi][j];
                g->in_elems[k] = (size_t)g->passes[pi]->m[j].in_elems;
                g->res_elems[k] = (size_t)g->passes[pi]->m[j].res_elems;
            }
        for (int k = 0; k < n; ++k) {
            g->in_off[k] = g->nin; g->nin += g->in_elems[k];
            g->res_off[k] = g->nres; g->nres += g->res_elems[k];
        }
        // every pass's launches, in order, in one graph
        e = cudaStreamSynchronize(g->stream);
        cudaGraph_t graph = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ei = cudaSuccess;
            for (tn_batch* b : g->passes)
                if (ei == cudaSuccess) ei = batch_issue(b, g->stream);
            e = cudaStreamEndCapture(g->stream, &graph);
            if (ei != cudaSuccess) e = ei;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) { g->gexec = nullptr; return cuda_status(e, "group graph"); }
        *out = owner.release();
        return TN_OK;
    } catch (const std::exception& ex) {
        set_error(ex.what());
        return TN_ERR_INVALID;
    }
}

tn_status tn_batch_group_destroy(tn_batch_group* g) {
    if (!g) return TN_ERR_INVALID;
    cudaStreamSynchronize(g->stream);
    group_free(g);
    return TN_OK;
}

tn_status tn_batch_group_info(const tn_batch_group* g, int* passes, size_t* arena_bytes, size_t* n_elems,
                              size_t* n_results, int64_t* launches) {
    if (!g) return TN_ERR_INVALID;
    if (passes) *passes = (int)g->passes.size();
    if (arena_bytes) *arena_bytes = g->arena_bytes;
    if (n_elems) *n_elems = g->nin;
    if (n_results) *n_results = g->nres;
    if (launches) {
        int64_t c = 0;
        for (const tn_batch* b : g->passes) c += (int64_t)b->launches.size() + 2;   // + init + final
        *launches = c;
    }
    return TN_OK;
}

tn_status tn_batch_group_set_tensors(tn_batch_group* g, const double* host, size_t n) {
    if (!g || !host || n != g->nin) { set_error("tensor count mismatch"); return TN_ERR_INVALID; }
    for (size_t pi = 0; pi < g->passes.size(); ++pi) {
        tn_batch* b = g->passes[pi];
        for (size_t j = 0; j < g->members[pi].size(); ++j) {
            const int k = g->members[pi][j];
            const cudaError_t e = cudaMemcpyAsync(b->buf + b->lay.in_off + (size_t)b->m[j].in_off * 8,
                                                  host + g->in_off[k], g->in_elems[k] * 8, cudaMemcpyHostToDevice,
                                                  g->stream);
            if (e != cudaSuccess) return cuda_status(e, "tensor upload");
        }
    }
    return cuda_status(cudaStreamSynchronize(g->stream), "tensor upload");
}

tn_status tn_batch_group_fill_random(tn_batch_group* g, uint64_t batch_seed) {
    try {
        if (!g) return TN_ERR_INVALID;
        // member k of the group takes the seed member k of one batch would
        std::vector<double> h(g->nin);
        for (int k = 0; k < g->n; ++k)
            fill_uniform(mix64g(batch_seed + (uint64_t)(k + 1) * kGammaG), h.data() + g->in_off[k], g->in_elems[k]);
        return tn_batch_group_set_tensors(g, h.data(), h.size());
    } catch (const std::exception& ex) {
        set_error(ex.what());
        return TN_ERR_INVALID;
    }
}

tn_status tn_batch_group_run(tn_batch_group* g, double J, const double* h) {
    if (!g || !h) return TN_ERR_INVALID;
    for (size_t pi = 0; pi < g->passes.size(); ++pi) {
        tn_batch* b = g->passes[pi];
        for (size_t j = 0; j < g->members[pi].size(); ++j) {
            b->h_final[j].J = J;
            b->h_final[j].h = h[g->members[pi][j]];
        }
        const cudaError_t e = cudaMemcpyAsync(b->buf + b->lay.final_off, b->h_final.data(),
                                              b->h_final.size() * sizeof(FinalTask), cudaMemcpyHostToDevice,
                                              g->stream);
        if (e != cudaSuccess) return cuda_status(e, "final table upload");
    }
    return cuda_status(cudaGraphLaunch(g->gexec, g->stream), "group graph launch");
}

tn_status tn_batch_group_results_host(tn_batch_group* g, double* host, size_t cap) {
    if (!g || !host || cap < g->nres) return TN_ERR_INVALID;
    std::vector<int> status(g->passes.size(), 0);
    cudaError_t e = cudaSuccess;
    for (size_t pi = 0; pi < g->passes.size() && e == cudaSuccess; ++pi) {
        tn_batch* b = g->passes[pi];
        for (size_t j = 0; j < g->members[pi].size() && e == cudaSuccess; ++j) {
            const int k = g->members[pi][j];
            e = cudaMemcpyAsync(host + g->res_off[k], b->buf + b->lay.res_off + (size_t)b->m[j].res_off * 8,
                                g->res_elems[k] * 8, cudaMemcpyDeviceToHost, g->stream);
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&status[pi], b->buf + b->lay.status_off, sizeof(int), cudaMemcpyDeviceToHost,
                                g->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return cuda_status(e, "result read");
    for (int s : status)
        if (s) { set_error("a bounded wait in a kernel timed out"); return TN_ERR_TIMEOUT; }
    return TN_OK;
}

}  // extern "C"
