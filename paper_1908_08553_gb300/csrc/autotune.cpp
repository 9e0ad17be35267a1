// Autotuner: for a lattice shape (L, W, D), a precision and a work kind, time
// every applicable combination of the program builder's choices (Knobs) on a
// batch of copies of that shape and keep the fastest in a table keyed on the
// shape.  Every batch and lattice created afterwards takes its programs with
// the table's choice for its shape, so a lattice is contracted the same way
// (and gives the same bits) alone, in any batch and when served.  The knobs
// are all exact reformulations; only speed differs.
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include "runtime.h"

namespace tn {

namespace {

struct TuneEntry {
    int knobs = kDefaultKnobs;
    double best_ms = 0.0, default_ms = 0.0;
    int copies = 0, candidates = 0;
};

using TuneKey = std::tuple<int, int, int, int, int>;   // L, W, D, precision, work
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;

// Knob combinations that change this shape's program (the default first).
std::vector<int> candidates(int D, tn_precision prec, tn_work work) {
    std::vector<int> bits;   // knob bits that apply
    const bool fp32_store = prec != TN_FP64;
    const bool tc = prec == TN_BF16X3 || prec == TN_BF16X6;
    if (D == 3) bits.push_back(4);              // factor_d3 (off: tensor-core D = 3 absorption when tc)
    if (fp32_store && D <= 2 && work != TN_WORK_NORM) bits.push_back(2);   // site_triple
    if (fp32_store && D == 2 && work != TN_WORK_NORM) bits.push_back(1);   // fuse_pairs
    if (tc) bits.push_back(8);                                             // tc_products
    if (tc) bits.push_back(16);                                            // tc_small
    // every combination of the applicable bits flipped from the default
    // (tc_small only matters with tc_products)
    std::vector<int> out{kDefaultKnobs};
    for (int mask = 1; mask < (1 << bits.size()); ++mask) {
        int code = kDefaultKnobs;
        for (size_t b = 0; b < bits.size(); ++b)
            if (mask & (1 << b)) code ^= bits[b];
        if ((code & 16) && !(code & 8)) continue;
        out.push_back(code);
    }
    return out;
}

}  // namespace

Knobs tuned_knobs(int L, int W, int D, tn_precision prec, tn_work work) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(L, W, D, (int)prec, (int)work));
    return Knobs::from_code(it == g_tune.end() ? kDefaultKnobs : it->second.knobs);
}

}  // namespace tn

using namespace tn;

extern "C" {

tn_status tn_autotune(tn_ctx* ctx, int n, const int* L, const int* W, const int* D, tn_precision prec,
                      tn_work work, int reps, size_t max_bytes) {
    try {
        if (!ctx || n <= 0 || !L || !W || !D || reps < 1 || prec < TN_FP64 || prec > TN_BF16X6 ||
            !(work == TN_WORK_NORM || work == TN_WORK_ENERGY)) {
            set_error("bad autotune arguments");
            return TN_ERR_INVALID;
        }
        if (ctx->device < 0) { set_error("context has no device"); return TN_ERR_NO_DEVICE; }
        if (max_bytes == 0) max_bytes = size_t(4) << 30;
        cudaSetDevice(ctx->device);
        std::map<std::tuple<int, int, int>, int> shapes;
        for (int k = 0; k < n; ++k) shapes[std::make_tuple(L[k], W[k], D[k])] = 1;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        tn_status result = TN_OK;
        for (const auto& sh : shapes) {
            const int l = std::get<0>(sh.first), w = std::get<1>(sh.first), d = std::get<2>(sh.first);
            // copies of the shape filling at most max_bytes (between 1 and 64)
            tn_batch* probe = nullptr;
            size_t fp = 0;
            tn_status st = batch_create(ctx, 1, &l, &w, &d, prec, TN_SCHED_AUTO, work, false, &probe, &fp);
            if (probe) batch_destroy(probe);
            if (st != TN_OK) { result = st; break; }
            if (fp > max_bytes) continue;                 // too large to tune within the limit
            const int copies = (int)std::max<size_t>(1, std::min<size_t>(64, max_bytes / std::max<size_t>(fp, 1)));
            std::vector<int> Ls(copies, l), Ws(copies, w), Ds(copies, d);
            std::vector<double> hs(copies, 3.04);
            TuneEntry best;
            best.copies = copies;
            const auto cands = candidates(d, prec, work);
            best.candidates = (int)cands.size();
            double best_ms = -1.0;
            for (int code : cands) {
                BatchOpts opts;
                opts.knobs = code;
                tn_batch* b = nullptr;
                st = batch_create(ctx, copies, Ls.data(), Ws.data(), Ds.data(), prec, TN_SCHED_AUTO, work, true, &b,
                                  nullptr, &opts);
                if (st != TN_OK) { result = st; break; }
                st = tn_batch_fill_random(b, 12345);
                for (int k = 0; k < copies && st == TN_OK; ++k) { b->h_final[k].J = 1.0; b->h_final[k].h = hs[k]; }
                if (st == TN_OK) st = batch_run(b, b->stream);     // capture + warm-up
                if (st == TN_OK) st = cuda_status(cudaStreamSynchronize(b->stream), "autotune warm-up");
                float ms = 0.0f;
                if (st == TN_OK) {
                    cudaEventRecord(e0, b->stream);
                    for (int r = 0; r < reps && st == TN_OK; ++r) st = batch_run(b, b->stream);
                    cudaEventRecord(e1, b->stream);
                    if (st == TN_OK) st = cuda_status(cudaEventSynchronize(e1), "autotune timing");
                    if (st == TN_OK) cudaEventElapsedTime(&ms, e0, e1);
                }
                batch_destroy(b);
                if (st != TN_OK) { result = st; break; }
                const double per = ms / reps;
                if (code == kDefaultKnobs) best.default_ms = per;
                // a candidate replaces the current choice only if it is 2% faster
                if (best_ms < 0.0 || per < 0.98 * best_ms) { best_ms = per; best.knobs = code; }
            }
            if (result != TN_OK) break;
            best.best_ms = best_ms;
            std::lock_guard<std::mutex> g(g_tune_mu);
            g_tune[std::make_tuple(l, w, d, (int)prec, (int)work)] = best;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return result;
    } catch (const std::exception& ex) {
        set_error(ex.what());
        return TN_ERR_INVALID;
    }
}

tn_status tn_autotune_lookup(int L, int W, int D, tn_precision prec, tn_work work, int* knobs, double* best_ms,
                             double* default_ms, int* tuned) {
    if (!knobs) return TN_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(L, W, D, (int)prec, (int)work));
    const bool found = it != g_tune.end();
    *knobs = found ? it->second.knobs : kDefaultKnobs;
    if (best_ms) *best_ms = found ? it->second.best_ms : 0.0;
    if (default_ms) *default_ms = found ? it->second.default_ms : 0.0;
    if (tuned) *tuned = found ? 1 : 0;
    return TN_OK;
}

tn_status tn_autotune_set(int L, int W, int D, tn_precision prec, tn_work work, int knobs) {
    if (knobs < 0 || knobs > kMaxKnobs || L < 1 || W < 1 || D < 1) return TN_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_tune_mu);
    TuneEntry& e = g_tune[std::make_tuple(L, W, D, (int)prec, (int)work)];
    e.knobs = knobs;
    return TN_OK;
}

tn_status tn_autotune_clear(void) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune.clear();
    return TN_OK;
}

tn_status tn_autotune_save(const char* path) {
    if (!path) return TN_ERR_INVALID;
    FILE* f = std::fopen(path, "w");
    if (!f) { set_error("cannot open the tuning file for writing"); return TN_ERR_INVALID; }
    std::lock_guard<std::mutex> g(g_tune_mu);
    std::fprintf(f, "# L W D precision work knobs best_ms default_ms copies candidates\n");
    for (const auto& kv : g_tune) {
        const auto& k = kv.first;
        const auto& e = kv.second;
        std::fprintf(f, "%d %d %d %d %d %d %.6f %.6f %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k),
                     std::get<3>(k), std::get<4>(k), e.knobs, e.best_ms, e.default_ms, e.copies, e.candidates);
    }
    std::fclose(f);
    return TN_OK;
}

tn_status tn_autotune_load(const char* path) {
    if (!path) return TN_ERR_INVALID;
    FILE* f = std::fopen(path, "r");
    if (!f) { set_error("cannot open the tuning file"); return TN_ERR_INVALID; }
    char line[256];
    std::map<TuneKey, TuneEntry> t;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#') continue;
        int l, w, d, p, wk, kn, cp, cd;
        double bm, dm;
        if (std::sscanf(line, "%d %d %d %d %d %d %lf %lf %d %d", &l, &w, &d, &p, &wk, &kn, &bm, &dm, &cp, &cd) != 10 ||
            kn < 0 || kn > kMaxKnobs) {
            std::fclose(f);
            set_error("malformed tuning file");
            return TN_ERR_INVALID;
        }
        TuneEntry e;
        e.knobs = kn; e.best_ms = bm; e.default_ms = dm; e.copies = cp; e.candidates = cd;
        t[std::make_tuple(l, w, d, p, wk)] = e;
    }
    std::fclose(f);
    std::lock_guard<std::mutex> g(g_tune_mu);
    for (const auto& kv : t) g_tune[kv.first] = kv.second;
    return TN_OK;
}

}  // extern "C"
