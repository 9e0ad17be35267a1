// Host runtime objects behind the C-ABI handles.
#pragma once

#include <atomic>
#include <condition_variable>
#include <deque>
#include <string>
#include <thread>
#include <unordered_map>

#include <cuda_runtime.h>

#include "tn_internal.h"
#include "tn_kernels.h"

namespace tn {

void set_error(const std::string& msg);

enum Family { FAM_ABSORB = 0, FAM_ABSORB_DOT = 1, FAM_GEMM = 2, FAM_TC = 3, FAM_OTHER = 4, FAM_PAIR = 5 };
constexpr int kFamilies = 6;

struct KStat {
    int64_t launches = 0;
    double ms = 0, bytes = 0, macs = 0;
};

struct Server;

// One grouped kernel launch of a batch run.
struct Launch {
    int kind = 0;         // OpKind
    int dt = 0;
    int K = 0, N = 0;
    int variant = 0;      // absorption kernel variant (see launch_absorb)
    size_t task_off = 0;  // bytes into the task region
    size_t map_off = 0;   // bytes into the task region of the block -> task table (0: none)
    int ntasks = 0;
    long long nblocks = 0;
    double bytes = 0, macs = 0;
};

struct Member {
    std::shared_ptr<const Program> pg;
    int L = 0, W = 0, D = 0;
    int64_t in_elems = 0, in_off = 0;   // FP64 entries
    int64_t arena_off = 0;              // bytes into the arena region
    int64_t slot_base = 0;
    int64_t res_off = 0, res_elems = 0; // doubles
};

// Byte layout of a batch's single device buffer.
struct Layout {
    size_t in_off = 0, arena_off = 0, slots_off = 0, part_off = 0, res_off = 0;
    size_t tasks_off = 0, status_off = 0, final_off = 0, ints_off = 0, ones_off = 0, total = 0;
    int64_t nslots = 0, npart = 0, nres = 0, nin = 0, nones = 0, nints = 0;
    size_t task_bytes = 0;
};

}  // namespace tn

struct tn_ctx {
    int device = -1;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool profiling = false;
    std::atomic<int> inject_timeouts{0};   // host-side fault injection (tn_ctx_inject_wait_timeout)
    tn::KStat stats[tn::kFamilies];
    std::mutex mu;          // guards stats and the server
    tn::Server* server = nullptr;
};

struct tn_batch {
    tn_ctx* ctx = nullptr;
    int dt = 1;
    tn_work work = TN_WORK_ENERGY;
    tn_schedule sched = TN_SCHED_AUTO;
    std::vector<tn::Member> m;
    tn::Layout lay;
    char* buf = nullptr;
    std::vector<tn::Launch> launches;
    std::vector<tn::FinalTask> h_final;
    std::vector<double> h_h;
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;
    cudaStream_t stream = nullptr;    // ctx stream unless the server assigns one
    bool async_alloc = false;         // buffer from the stream-ordered pool (served batches)
    std::vector<char> h_tasks;        // host copies of the uploaded tables
    std::vector<int> h_ints;
    std::vector<tn::ConstOne> h_ones;
    bool arena_external = false;      // the arena lives outside buf (shared by the passes of a group)
    char* ext_arena = nullptr;
    size_t arena_bytes = 0;           // the members' arena, wherever it lives
};

struct tn_lattice {
    tn_ctx* ctx = nullptr;
    int L = 0, W = 0, D = 0;
    std::vector<double> host;        // input layout of the lattice's programs
    bool cplx = false;               // complex site tensors (host: per site real parts, then imaginary)
    std::map<std::tuple<int, int, int>, tn_batch*> cache;   // (prec, sched, work) -> 1-member batch
};

namespace tn {
struct BatchOpts {
    cudaStream_t stream = nullptr;   // default: the context's stream
    bool async_alloc = false;        // cudaMallocAsync / cudaFreeAsync on that stream
    bool use_graph = true;           // capture the launch sequence on the first run
    int knobs = -1;                  // program knobs (Knobs::code); -1: the tuning table's choice
    std::vector<int> member_knobs;   // per member instead of knobs (when not empty)
    std::shared_ptr<const Program> program;   // every member runs this program (its shape must match)
    bool complex_sites = false;      // complex site tensors (every member)
    bool arena_external = false;     // no arena in the batch buffer: the tensors live in ext_arena
    char* ext_arena = nullptr;       // (null when only sizes are computed)
    size_t ext_arena_bytes = 0;
};
tn_status batch_create(tn_ctx* ctx, int n, const int* L, const int* W, const int* D,
                       tn_precision prec, tn_schedule sched, tn_work work, bool alloc,
                       tn_batch** out, size_t* bytes, const BatchOpts* opts = nullptr);
std::shared_ptr<const Program> program_cached(int L, int W, int D, tn_schedule sched, tn_precision prec,
                                              tn_work work, int knobs_code = -1, bool cplx = false);
tn_status batch_run(tn_batch* b, cudaStream_t st);
// The kernel launches of one run (no table upload): what a graph captures.
cudaError_t batch_issue(tn_batch* b, cudaStream_t st);
void batch_destroy(tn_batch* b);
tn_status cuda_status(cudaError_t e, const char* what);
void preload_kernels(int device);
void server_stop(tn_ctx* ctx);
}  // namespace tn
