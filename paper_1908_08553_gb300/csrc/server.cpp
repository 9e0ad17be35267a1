// Request server: tn_submit / tn_poll / tn_wait with continuous batching.
//
// A scheduler thread per context keeps a FIFO of submitted jobs.  Each job's
// device time is estimated at submit from its contraction program (multiply-
// adds and bytes of every pairwise contraction), which sorts it into one of two
// classes.  Light jobs are batched: whenever one of the high-priority streams
// is free and the HBM budget left by running batches allows, the scheduler
// takes the light jobs in FIFO order with the first one's precision whose
// exact footprints fit, builds one batch from them (one device buffer from the
// stream-ordered pool, grouped launches), uploads their tensors, runs it on
// that stream and queues the read-back of the results.  Heavy jobs (seconds of
// work, tens of GB) run alone, one per low-priority stream, so a light job
// never waits for a heavy one to finish: its blocks are scheduled ahead of the
// heavy job's on the SMs.  When a batch's completion event fires its results
// go to the jobs, its memory returns to the budget, and jobs that were waiting
// for memory are admitted.  A job whose footprint alone exceeds the budget is
// refused at submit time (TN_ERR_OVER_BUDGET).  Every member's results depend
// only on its own tasks (shape-fixed tiles, index-ordered reductions), so a
// job gives the same bits alone, in any mix and on either stream class.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "runtime.h"

namespace tn {

void fill_uniform(uint64_t seed, double* out, size_t n);
tn_status result_from_array(const double* r, int L, int W, tn_precision prec, const Plan& p, tn_result* out);

namespace {

using Clock = std::chrono::steady_clock;

struct SJob {
    uint64_t ticket = 0;
    int L = 0, W = 0, D = 0;
    tn_precision prec = TN_FP32;
    double J = 1.0, h = 0.0;
    std::vector<double> tensors;
    size_t footprint = 0;
    double est_s = 0.0;         // estimated device time
    bool heavy = false;
    int state = 0;              // 0 pending, 1 running, 2 finished
    tn_status status = TN_OK;
    std::vector<double> result;
    std::shared_ptr<const Program> pg;
};

struct SBatch {
    tn_batch* b = nullptr;
    std::vector<SJob*> jobs;
    cudaEvent_t done = nullptr;
    int slot = -1;
};

constexpr int kLightStreams = 6;              // high priority, batched light jobs
constexpr int kHeavyStreams = 2;              // low priority, one heavy job each
constexpr int kStreams = kLightStreams + kHeavyStreams;
constexpr int kMaxMembers = 256;
constexpr double kHeavySeconds = 0.02;        // estimated device time that makes a job heavy
// result doubles of one served member at most: header, <X_k>, <Z_i Z_j>, <Z_k>
// of a 16 x 16 lattice
constexpr size_t kMaxResult = kResultHeader + 256 + 2 * 16 * 15 + 256;

// Device time of a job from its program: multiply-adds at a sustained rate of
// the precision's arithmetic plus bytes at a sustained HBM rate, plus launch
// latency per wave.  Only orders jobs; nothing depends on its accuracy.
double estimate_seconds(const Program& pg, tn_precision prec) {
    double macs = 0.0, bytes = 0.0;
    for (const Op& op : pg.ops) { macs += (double)op.macs; bytes += (double)op.bytes; }
    const double rate = prec == TN_FP64 ? 5e11 : (pg.nsplit ? 1e14 : 2e13);
    return macs / rate + bytes / 3e12 + 5e-6 * pg.n_levels;
}

}  // namespace

struct Server {
    tn_ctx* ctx = nullptr;
    std::mutex mu;
    std::condition_variable cv;        // scheduler wake-up
    std::condition_variable cv_done;   // job completion
    std::deque<SJob*> pending;
    std::unordered_map<uint64_t, SJob*> jobs;
    std::vector<SBatch> inflight;
    cudaStream_t streams[kStreams] = {};
    bool busy[kStreams] = {};
    double* pinned[kStreams] = {};     // result read-back buffers
    size_t pinned_n[kStreams] = {};
    std::thread th;
    bool stop = false;
    uint64_t next = 1;

    void loop();
    void retire_locked();
    bool admit(std::unique_lock<std::mutex>& lk);
};

void Server::retire_locked() {
    for (auto it = inflight.begin(); it != inflight.end();) {
        const cudaError_t q = cudaEventQuery(it->done);
        if (q == cudaErrorNotReady) { ++it; continue; }
        const double* r = pinned[it->slot];
        // the batch's status word rides behind its results: nonzero when a
        // bounded wait inside one of its kernels ran out (the results are then
        // incomplete), so every job of the batch reports the timeout
        int wait_status = 0;
        if (q == cudaSuccess) std::memcpy(&wait_status, r + it->b->lay.nres, sizeof(int));
        for (size_t k = 0; k < it->jobs.size(); ++k) {
            SJob* j = it->jobs[k];
            const Member& mb = it->b->m[k];
            if (q == cudaSuccess && wait_status) {
                j->status = TN_ERR_TIMEOUT;
            } else if (q == cudaSuccess) {
                j->result.assign(r + mb.res_off, r + mb.res_off + mb.res_elems);
                j->status = TN_OK;
            } else {
                j->status = cuda_status(q, "served batch");
            }
            j->state = 2;
        }
        cudaEventDestroy(it->done);
        batch_destroy(it->b);
        busy[it->slot] = false;
        it = inflight.erase(it);
        cv_done.notify_all();
    }
}

bool Server::admit(std::unique_lock<std::mutex>& lk) {
    if (pending.empty()) return false;
    const size_t left = ctx->budget > ctx->used.load() ? ctx->budget - ctx->used.load() : 0;
    auto free_slot = [&](int s0, int s1) {
        for (int s = s0; s < s1; ++s)
            if (!busy[s]) return s;
        return -1;
    };
    std::vector<SJob*> take;
    int slot = free_slot(0, kLightStreams);
    if (slot >= 0) {
        // light jobs in FIFO order with the first one's precision that fit the
        // budget left (stopping at the first that does not: no overtaking there)
        int prec = -1;
        size_t sum = 0;
        for (SJob* j : pending) {
            if (j->heavy) continue;
            if (prec < 0) prec = j->prec;
            if ((int)j->prec != prec || (int)take.size() >= kMaxMembers || sum + j->footprint > left) break;
            sum += j->footprint;
            take.push_back(j);
        }
    }
    if (take.empty()) {
        // the first heavy job, alone, if a low-priority stream and its memory are free
        slot = free_slot(kLightStreams, kStreams);
        if (slot < 0) return false;
        for (SJob* j : pending)
            if (j->heavy) {
                if (j->footprint <= left) take.push_back(j);
                break;
            }
        if (take.empty()) return false;   // it waits for memory to free up
    }
    for (SJob* j : take) pending.erase(std::find(pending.begin(), pending.end(), j));
    for (SJob* j : take) j->state = 1;
    busy[slot] = true;
    lk.unlock();

    std::vector<int> L, W, D;
    std::vector<double> in;
    for (SJob* j : take) {
        L.push_back(j->L); W.push_back(j->W); D.push_back(j->D);
        in.insert(in.end(), j->tensors.begin(), j->tensors.end());
    }
    BatchOpts opts;
    opts.stream = streams[slot];
    opts.async_alloc = true;
    opts.use_graph = false;
    tn_batch* b = nullptr;
    tn_status st = batch_create(ctx, (int)take.size(), L.data(), W.data(), D.data(), take[0]->prec, TN_SCHED_AUTO,
                                TN_WORK_ENERGY, true, &b, nullptr, &opts);
    cudaEvent_t ev = nullptr;
    if (st == TN_OK) {
        for (size_t k = 0; k < take.size(); ++k) {
            b->h_final[k].J = take[k]->J;
            b->h_final[k].h = take[k]->h;
        }
        st = cuda_status(cudaMemcpyAsync(b->buf + b->lay.in_off, in.data(), in.size() * 8,
                                         cudaMemcpyHostToDevice, b->stream), "served upload");
        if (st == TN_OK) st = batch_run(b, b->stream);
        // read-back buffer: the results, then one double holding the status word
        // (allocated once per slot for the largest batch: freeing pinned memory
        // would synchronise the whole device, stalling the scheduler behind
        // every running job)
        const size_t need = (size_t)b->lay.nres + 1;
        if (st == TN_OK && pinned_n[slot] < need) {
            set_error("no pinned read-back buffer for this batch");
            st = TN_ERR_OOM;
        }
        if (st == TN_OK)
            st = cuda_status(cudaMemcpyAsync(pinned[slot], b->buf + b->lay.res_off, (size_t)b->lay.nres * 8,
                                             cudaMemcpyDeviceToHost, b->stream), "served read-back");
        if (st == TN_OK)
            st = cuda_status(cudaMemcpyAsync(pinned[slot] + b->lay.nres, b->buf + b->lay.status_off, sizeof(int),
                                             cudaMemcpyDeviceToHost, b->stream), "served status read-back");
        if (st == TN_OK) st = cuda_status(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        if (st == TN_OK) st = cuda_status(cudaEventRecord(ev, b->stream), "event record");
    }
    lk.lock();
    if (st != TN_OK) {
        if (ev) cudaEventDestroy(ev);
        if (b) batch_destroy(b);
        busy[slot] = false;
        if (st == TN_ERR_OVER_BUDGET) {
            // the estimate was optimistic: put the jobs back at the head
            for (auto it = take.rbegin(); it != take.rend(); ++it) { (*it)->state = 0; pending.push_front(*it); }
            return false;
        }
        for (SJob* j : take) { j->status = st; j->state = 2; }
        cv_done.notify_all();
        return true;
    }
    SBatch sb;
    sb.b = b;
    sb.jobs = take;
    sb.done = ev;
    sb.slot = slot;
    inflight.push_back(sb);
    return true;
}

void Server::loop() {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        retire_locked();
        bool progressed = false;
        while (admit(lk)) progressed = true;
        if (stop && pending.empty() && inflight.empty()) break;
        if (!progressed) cv.wait_for(lk, std::chrono::microseconds(inflight.empty() ? 2000 : 50));
    }
}

namespace {

Server* get_server(tn_ctx* ctx, bool create) {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (!ctx->server && create) {
        auto* s = new Server();
        s->ctx = ctx;
        cudaSetDevice(ctx->device);
        // light batches on the highest stream priority, heavy jobs on the lowest
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        for (int k = 0; k < kStreams; ++k)
            cudaStreamCreateWithPriority(&s->streams[k], cudaStreamNonBlocking, k < kLightStreams ? greatest : least);
        // keep freed batch memory in the pool instead of returning it to the driver
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
            uint64_t thr = ctx->budget;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        for (int k = 0; k < kStreams; ++k) {
            const size_t n = (size_t)kMaxMembers * kMaxResult + 1;
            if (cudaMallocHost(reinterpret_cast<void**>(&s->pinned[k]), n * 8) == cudaSuccess) s->pinned_n[k] = n;
            else s->pinned[k] = nullptr;
        }
        s->th = std::thread([s] { s->loop(); });
        ctx->server = s;
    }
    return ctx->server;
}

}  // namespace

void server_stop(tn_ctx* ctx) {
    Server* s = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        s = ctx->server;
        ctx->server = nullptr;
    }
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    for (int k = 0; k < kStreams; ++k) {
        if (s->streams[k]) { cudaStreamSynchronize(s->streams[k]); cudaStreamDestroy(s->streams[k]); }
        if (s->pinned[k]) cudaFreeHost(s->pinned[k]);
    }
    for (auto& kv : s->jobs) delete kv.second;
    delete s;
}

}  // namespace tn

using namespace tn;

extern "C" {

tn_status tn_submit(tn_ctx* ctx, const tn_job* job, uint64_t* ticket) {
    try {
        if (!ctx || !job || !ticket) return TN_ERR_INVALID;
        if (ctx->device < 0) { set_error("context has no device"); return TN_ERR_NO_DEVICE; }
        if (job->L < 1 || job->L > 16 || job->W < 1 || job->W > 16 || job->D < 1 || job->D > 4 ||
            job->precision < TN_FP64 || job->precision > TN_BF16X6) {
            set_error("bad job");
            return TN_ERR_INVALID;
        }
        auto j = std::make_unique<SJob>();
        j->L = job->L; j->W = job->W; j->D = job->D;
        j->prec = job->precision;
        j->J = job->J; j->h = job->h;
        const size_t n = tn_lattice_elems(j->L, j->W, j->D);
        j->tensors.resize(n);
        if (job->tensors) std::memcpy(j->tensors.data(), job->tensors, n * sizeof(double));
        else fill_uniform(job->seed, j->tensors.data(), n);
        tn_batch* probe = nullptr;
        tn_status st = batch_create(ctx, 1, &j->L, &j->W, &j->D, j->prec, TN_SCHED_AUTO, TN_WORK_ENERGY, false,
                                    &probe, &j->footprint);
        if (probe) {
            j->est_s = estimate_seconds(*probe->m[0].pg, j->prec);
            j->heavy = j->est_s > kHeavySeconds;
            delete probe;
        }
        if (st != TN_OK) return st;
        if (j->footprint > ctx->budget) {
            set_error("job footprint " + std::to_string(j->footprint) + " B exceeds the budget");
            return TN_ERR_OVER_BUDGET;
        }
        Server* s = get_server(ctx, true);
        {
            std::lock_guard<std::mutex> g(s->mu);
            j->ticket = s->next++;
            *ticket = j->ticket;
            s->jobs[j->ticket] = j.get();
            s->pending.push_back(j.release());
        }
        s->cv.notify_one();
        return TN_OK;
    } catch (const std::exception& e) {
        set_error(e.what());
        return TN_ERR_INVALID;
    }
}

static tn_status take_result(Server* s, uint64_t ticket, tn_result* out, std::unique_lock<std::mutex>& lk) {
    (void)lk;
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) { set_error("unknown ticket"); return TN_ERR_INVALID; }
    SJob* j = it->second;
    if (j->state < 2) return TN_NOT_READY;
    tn_status st = j->status;
    if (st == TN_OK && out) {
        const Plan p = plan_choose(j->L, j->W, j->D, TN_SCHED_AUTO, TN_WORK_ENERGY);
        st = result_from_array(j->result.data(), j->L, j->W, j->prec, p, out);
    }
    s->jobs.erase(it);
    delete j;
    return st;
}

tn_status tn_poll(tn_ctx* ctx, uint64_t ticket, tn_result* out) {
    if (!ctx) return TN_ERR_INVALID;
    Server* s = get_server(ctx, false);
    if (!s) { set_error("unknown ticket"); return TN_ERR_INVALID; }
    std::unique_lock<std::mutex> lk(s->mu);
    return take_result(s, ticket, out, lk);
}

tn_status tn_wait(tn_ctx* ctx, uint64_t ticket, double timeout_s, tn_result* out) {
    if (!ctx || timeout_s < 0) return TN_ERR_INVALID;
    Server* s = get_server(ctx, false);
    if (!s) { set_error("unknown ticket"); return TN_ERR_INVALID; }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) { set_error("unknown ticket"); return TN_ERR_INVALID; }
    SJob* j = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                              std::chrono::duration<double>(timeout_s));
    if (!s->cv_done.wait_until(lk, deadline, [j] { return j->state >= 2; })) {
        set_error("deadline passed before the job finished");
        return TN_ERR_TIMEOUT;
    }
    return take_result(s, ticket, out, lk);
}

}  // extern "C"
