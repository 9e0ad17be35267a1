// Batch runtime: lays out one device buffer per batch (site inputs, tensor
// arena, rescaling slots, dot partials, results, task tables), groups every
// member's operations wave by wave into grouped launches, and replays the
// launch sequence as a CUDA graph.
#include <algorithm>
#include <cstring>

#include "runtime.h"

namespace tn {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }
const char* last_error() { return g_err.c_str(); }

tn_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TN_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? TN_ERR_OOM : TN_ERR_CUDA;
}

namespace {

constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct OpRef {
    int member, op;
};

int family_of(int kind) {
    switch (kind) {
        case OP_ABSORB: return FAM_ABSORB;
        case OP_ABSORB_DOT: return FAM_ABSORB_DOT;
        case OP_ABSORB2: case OP_ABSORB2_DOT: return FAM_PAIR;
        case OP_TC_SPLIT: return FAM_OTHER;
        case OP_GEMM: case OP_GEMM_DOT: return FAM_GEMM;
        case OP_TC_GEMM: case OP_TC_GEMM_DOT: return FAM_TC;
        default: return FAM_OTHER;
    }
}

// Build every launch and its task table.  With base == nullptr only sizes are
// computed (footprint); otherwise task structs hold absolute device pointers.
long long absorb_tiles_any(int var, long long P, long long S, int K, int N) {
    if (var == kAbsorbTwoPass) return absorb_2pass_tiles(P, S);
    if (var >= 20) return absorb_tiles_v(var - 20, P, S, K, N);   // triple dot of variants 1 / 2
    if (var >= 10) return absorb_tiles_v(var - 10, P, S, K, N);   // dual dot of variants 1 / 2
    if (var >= 3) return tc_absorb_tiles(P, S);
    return absorb_tiles_v(var, P, S, K, N);
}

void materialize(tn_batch* b, char* base, std::vector<char>* tasks_out, std::vector<int>* ints_out,
                 std::vector<ConstOne>* ones_out) {
    Layout& lay = b->lay;
    const int esize = b->dt == 0 ? 8 : 4;
    // --- regions that do not depend on tasks
    int64_t nin = 0, nslots = 0, nres = 0;
    size_t arena = 0;
    for (auto& mb : b->m) {
        mb.in_off = nin;
        mb.in_elems = mb.pg->site_offset.back();
        nin += mb.in_elems;
        mb.arena_off = (int64_t)arena;
        arena += up((size_t)mb.pg->arena_bytes);
        mb.slot_base = nslots;
        nslots += mb.pg->n_slots;
        mb.res_off = nres;
        mb.res_elems = kResultHeader + (int64_t)mb.pg->sx_slot.size() + (int64_t)mb.pg->zz_slot.size() +
                       (int64_t)mb.pg->sz_slot.size() + (int64_t)mb.pg->sy_slot.size();
        nres += mb.res_elems;
    }
    lay.nin = nin;
    lay.nslots = nslots;
    lay.nres = nres;
    // --- group operations: (level, kind, K, N, variant) -> op refs (member-major order)
    std::map<std::tuple<int, int, int, int, int>, std::vector<OpRef>> groups;
    int64_t npart = 0;
    for (int mi = 0; mi < (int)b->m.size(); ++mi) {
        const Program& pg = *b->m[mi].pg;
        for (int oi = 0; oi < (int)pg.ops.size(); ++oi) {
            const Op& op = pg.ops[oi];
            int K = 0, N = 0, var = 0;
            if (op.kind == OP_ABSORB || op.kind == OP_ABSORB_DOT) {
                K = op.K; N = op.N;
                // 0..2: SIMT (generic, 4 positions along s, 4 along p); 3 / 4: tensor
                // cores with 2 / 3 split planes; +10: dual dot; +20: triple dot
                var = op.nsplit ? 1 + op.nsplit : absorb_variant(b->dt, op.P, op.S, op.K, op.N);
                if (op.E3 >= 0) var += 20;
                else if (op.E2 >= 0) var += 10;
                if (op.factored) var = kAbsorbTwoPass;   // 30: ket pass then bra pass (D = 3)
            } else if (op.kind == OP_ABSORB2 || op.kind == OP_ABSORB2_DOT) {
                K = op.K; N = op.N;
            } else if (op.kind == OP_GEMM || op.kind == OP_GEMM_DOT) {
                var = gemm_variant(b->dt, op.gm, op.gn, op.gk, op.sam, op.sak, op.sbk, op.sbn);
            } else if (op.kind == OP_TC_GEMM || op.kind == OP_TC_GEMM_DOT) {
                // short k range (+10000), planes, tile width
                var = (op.Kp <= kTcShortK ? 10000 : 0) + op.nsplit * 1000 +
                      tc_gemm_bn(op.nsplit, op.kind == OP_TC_GEMM_DOT, op.gn, op.Kp);
            }
            groups[std::make_tuple(op.level, (int)op.kind, K, N, var)].push_back({mi, oi});
        }
    }
    // --- device pointers of the fixed regions
    lay.in_off = 0;
    b->arena_bytes = arena;
    lay.arena_off = up(lay.in_off + (size_t)nin * 8);
    lay.slots_off = b->arena_external ? lay.arena_off : up(lay.arena_off + arena);
    auto ptr = [&](size_t off) -> char* { return base ? base + off : nullptr; };
    Slot* slots_base = reinterpret_cast<Slot*>(ptr(lay.slots_off));
    (void)slots_base;
    // partial offsets are assigned while tasks are generated; region placed after slots
    std::vector<char> tasks;
    std::vector<int> ints;
    std::vector<ConstOne> ones;
    b->launches.clear();
    auto tensor_ptr = [&](int mi, int tid) -> void* {
        const Member& mb = b->m[mi];
        const Tensor& t = mb.pg->tensors[tid];
        if (!base) return nullptr;
        char* arena_base = b->arena_external ? b->ext_arena : base + lay.arena_off;
        return arena_base + mb.arena_off + t.offset;
    };
    auto slot_of = [&](int mi, int tid) -> int {
        return (int)(b->m[mi].slot_base + b->m[mi].pg->tensors[tid].slot);
    };
    // partial region placement needs npart first: count dot tiles
    for (auto& kv : groups) {
        const int kind = std::get<1>(kv.first);
        for (const OpRef& r : kv.second) {
            const Op& op = b->m[r.member].pg->ops[r.op];
            if (kind == OP_ABSORB_DOT) {
                const int var = std::get<4>(kv.first);
                npart += (1 + (op.E2 >= 0) + (op.E3 >= 0)) * absorb_tiles_any(var, op.P, op.S, op.K, op.N);
            }
            else if (kind == OP_GEMM_DOT) {
                int tn_;
                const int var = std::get<4>(kv.first);
                npart += gemm_tiles_v(var, op.gm, op.gn, &tn_) * gemm_ksplit(var, true, op.gk);
            }
            else if (kind == OP_DOT) npart += (op.gm + kDotPerBlock - 1) / kDotPerBlock;
            else if (kind == OP_ABSORB2_DOT) npart += absorb2_tiles(op.P, op.S);
            else if (kind == OP_TC_GEMM_DOT) {
                const int bn = std::get<4>(kv.first) % 1000;
                npart += ((op.gm + 127) / 128) * ((op.gn + bn - 1) / bn);   // one partial per tile
            }
        }
    }
    lay.npart = npart;
    lay.part_off = up(lay.slots_off + (size_t)nslots * sizeof(Slot));
    lay.res_off = up(lay.part_off + (size_t)npart * 8);
    lay.tasks_off = up(lay.res_off + (size_t)nres * 8);
    double* part_base = reinterpret_cast<double*>(ptr(lay.part_off));
    int64_t part_cur = 0;
    auto take_partial = [&](long long n) -> double* {
        double* p = part_base ? part_base + part_cur : nullptr;
        part_cur += n;
        return p;
    };
    // Tasks of one launch are packed back to back (the kernel indexes them as
    // an array of the task type); only the start of each launch is aligned.
    auto align_group = [&]() { tasks.resize((tasks.size() + 63) / 64 * 64); };
    auto append = [&](const void* src, size_t n) -> size_t {
        const size_t off = tasks.size();
        tasks.resize(off + n);
        std::memcpy(tasks.data() + off, src, n);
        return off;
    };
    for (auto& kv : groups) {
        const int kind = std::get<1>(kv.first);
        Launch L;
        L.kind = kind;
        L.dt = b->dt;
        L.K = std::get<2>(kv.first);
        L.N = std::get<3>(kv.first);
        L.variant = std::get<4>(kv.first);
        const auto& refs = kv.second;
        L.ntasks = (int)refs.size();
        long long tile = 0;
        align_group();
        size_t first = SIZE_MAX;
        std::vector<long long> starts;
        for (const OpRef& r : refs) {
            starts.push_back(tile);
            const Member& mb = b->m[r.member];
            const Program& pg = *mb.pg;
            const Op& op = pg.ops[r.op];
            L.bytes += op.bytes;
            L.macs += op.macs;
            size_t off = 0;
            if (kind == OP_SITEMAT) {
                SiteMatTask t{};
                t.A = base ? reinterpret_cast<const double*>(base + lay.in_off) + mb.in_off + pg.site_offset[op.site]
                           : nullptr;
                t.E = tensor_ptr(r.member, op.out);
                for (int k = 0; k < 4; ++k) { t.dims[k] = pg.site_dims[4 * op.site + k]; t.map[k] = op.map[k]; }
                t.phys = op.phys;
                t.slot_E = slot_of(r.member, op.out);
                t.K = op.K; t.N = op.N;
                t.factored = op.factored ? 1 : 0;
                // complex: the imaginary parts follow the real parts of the site
                t.Ai = (pg.cplx && t.A) ? t.A + (pg.site_offset[op.site + 1] - pg.site_offset[op.site]) / 2 : nullptr;
                off = append(&t, sizeof(t));
                tile += 1;
            } else if (kind == OP_ABSORB || kind == OP_ABSORB_DOT) {
                AbsorbTask t{};
                t.in = tensor_ptr(r.member, op.in);
                t.E = tensor_ptr(r.member, op.E);
                t.P = op.P; t.S = op.S; t.K = op.K; t.N = op.N;
                t.transE = op.transE ? 1 : 0;
                t.slot_in = slot_of(r.member, op.in);
                t.slot_E = slot_of(r.member, op.E);
                t.slot_out = slot_of(r.member, op.out);
                t.tile0 = tile;
                const long long nt = absorb_tiles_any(L.variant, op.P, op.S, op.K, op.N);
                t.ntiles = (int)nt;
                if (kind == OP_ABSORB_DOT) {
                    t.adj = tensor_ptr(r.member, op.adj);
                    t.slot_adj = slot_of(r.member, op.adj);
                    t.partial = take_partial((1 + (op.E2 >= 0) + (op.E3 >= 0)) * nt);
                    if (op.E2 >= 0) {
                        t.E2 = tensor_ptr(r.member, op.E2);
                        t.slot_E2 = slot_of(r.member, op.E2);
                        t.slot_out2 = slot_of(r.member, op.out2);
                    }
                    if (op.E3 >= 0) {
                        t.E3 = tensor_ptr(r.member, op.E3);
                        t.slot_E3 = slot_of(r.member, op.E3);
                        t.slot_out3 = slot_of(r.member, op.out3);
                    }
                } else {
                    t.out = tensor_ptr(r.member, op.out);
                }
                off = append(&t, sizeof(t));
                tile += nt;
            } else if (kind == OP_ABSORB2 || kind == OP_ABSORB2_DOT) {
                AbsorbTask t{};
                t.in = tensor_ptr(r.member, op.in);
                t.E = tensor_ptr(r.member, op.E);
                t.E2 = tensor_ptr(r.member, op.E2);
                t.P = op.P; t.S = op.S; t.K = op.K; t.N = op.N;
                t.slot_in = slot_of(r.member, op.in);
                t.slot_E = slot_of(r.member, op.E);
                t.slot_E2 = slot_of(r.member, op.E2);
                t.slot_out = slot_of(r.member, op.out);
                t.tile0 = tile;
                const long long nt = absorb2_tiles(op.P, op.S);
                t.ntiles = (int)nt;
                if (kind == OP_ABSORB2_DOT) {
                    t.adj = tensor_ptr(r.member, op.adj);
                    t.slot_adj = slot_of(r.member, op.adj);
                    t.partial = take_partial(nt);
                } else {
                    t.out = tensor_ptr(r.member, op.out);
                }
                off = append(&t, sizeof(t));
                tile += nt;
            } else if (kind == OP_GEMM || kind == OP_GEMM_DOT) {
                GemmTask t{};
                t.A = tensor_ptr(r.member, op.A);
                t.B = tensor_ptr(r.member, op.B);
                t.M = op.gm; t.N = op.gn; t.K = op.gk;
                t.sam = op.sam; t.sak = op.sak; t.sbk = op.sbk; t.sbn = op.sbn;
                t.slot_A = slot_of(r.member, op.A);
                t.slot_B = slot_of(r.member, op.B);
                t.slot_C = slot_of(r.member, op.out);
                int tn_ = 0;
                const long long ksp = gemm_ksplit(L.variant, kind == OP_GEMM_DOT, op.gk);
                const long long nt = gemm_tiles_v(L.variant, op.gm, op.gn, &tn_) * ksp;
                t.tiles_n = tn_;
                t.ntiles = (int)nt;
                t.ksplit = (int)ksp;
                t.kslice = ksp > 1 ? kGemmKSlice : op.gk;
                t.tile0 = tile;
                if (kind == OP_GEMM_DOT) {
                    t.Dm = tensor_ptr(r.member, op.C);
                    t.slot_D = slot_of(r.member, op.C);
                    t.partial = take_partial(nt);
                } else {
                    t.C = tensor_ptr(r.member, op.out);
                }
                off = append(&t, sizeof(t));
                tile += nt;
            } else if (kind == OP_TC_SPLIT) {
                TcSplitTask t{};
                t.src = tensor_ptr(r.member, op.A);
                t.dst = tensor_ptr(r.member, op.out);
                t.R = op.gm; t.Kd = op.gk; t.sr = op.sam; t.sk = op.sak;
                t.Rp = op.Rp; t.Kp = op.Kp;
                t.plane_bytes = op.Rp * op.Kp * 2;
                t.nsplit = op.nsplit;
                t.slot_src = slot_of(r.member, op.A);
                const long long nt = tc_split_tiles(op.Rp, op.Kp);
                t.ntiles = (int)nt;
                t.tile0 = tile;
                off = append(&t, sizeof(t));
                tile += nt;
            } else if (kind == OP_TC_GEMM || kind == OP_TC_GEMM_DOT) {
                TcGemmTask t{};
                t.A = tensor_ptr(r.member, op.A);
                t.B = tensor_ptr(r.member, op.B);
                const int bn = L.variant % 1000;
                const long long Ma = (op.gm + kTcRowPad - 1) / kTcRowPad * kTcRowPad;
                const long long Nb = (op.gn + kTcRowPad - 1) / kTcRowPad * kTcRowPad;
                t.a_plane_bytes = Ma * op.Kp * 2;
                t.b_plane_bytes = Nb * op.Kp * 2;
                t.M = op.gm; t.N = op.gn; t.Kp = op.Kp;
                t.slot_A = slot_of(r.member, op.A_src);
                t.slot_B = slot_of(r.member, op.B_src);
                t.slot_C = slot_of(r.member, op.out);
                t.tiles_m = (op.gm + 127) / 128;
                t.tiles_n = (int)((op.gn + bn - 1) / bn);
                // products fused with a dot keep the whole k range in one CTA (its
                // 512-term slices are pipelined inside, launch_tc_gemm_dot)
                const long long ksp = 1;
                t.ksplit = 1;
                t.kchunks = op.Kp / kTcChunk;
                const long long nt = t.tiles_m * t.tiles_n * ksp;
                t.ntiles = (int)nt;
                t.tile0 = tile;
                if (kind == OP_TC_GEMM_DOT) {
                    t.Dm = tensor_ptr(r.member, op.C);
                    t.slot_D = slot_of(r.member, op.C);
                    t.partial = take_partial(nt);
                } else {
                    t.C = tensor_ptr(r.member, op.out);
                }
                off = append(&t, sizeof(t));
                tile += nt;
            } else if (kind == OP_DOT) {
                DotTask t{};
                t.A = tensor_ptr(r.member, op.A);
                t.B = tensor_ptr(r.member, op.B);
                t.n = op.gm;
                t.slot_A = slot_of(r.member, op.A);
                t.slot_B = slot_of(r.member, op.B);
                t.slot_out = slot_of(r.member, op.out);
                const long long nt = (op.gm + kDotPerBlock - 1) / kDotPerBlock;
                t.ntiles = (int)nt;
                t.tile0 = tile;
                t.partial = take_partial(nt);
                off = append(&t, sizeof(t));
                tile += nt;
            }
            first = std::min(first, off);
        }
        L.task_off = first;
        L.nblocks = tile;
        // block -> task table for launches of many short blocks (saves each
        // block a dependent binary search over the task list)
        const bool mapped = ((kind == OP_ABSORB || kind == OP_ABSORB_DOT) && (L.variant <= 2 || L.variant >= 10)) ||   // SIMT variants
                            kind == OP_DOT || kind == OP_ABSORB2 || kind == OP_ABSORB2_DOT;
        if (mapped && L.ntasks > 8) {
            tasks.resize((tasks.size() + 15) / 16 * 16);
            L.map_off = tasks.size();
            tasks.resize(tasks.size() + (size_t)tile * sizeof(int));
            int* mp = reinterpret_cast<int*>(tasks.data() + L.map_off);
            for (size_t ti = 0; ti < starts.size(); ++ti) {
                const long long end = ti + 1 < starts.size() ? starts[ti + 1] : tile;
                for (long long k = starts[ti]; k < end; ++k) mp[k] = (int)ti;
            }
        }
        b->launches.push_back(L);
    }
    // const-one tensors
    for (int mi = 0; mi < (int)b->m.size(); ++mi) {
        const Program& pg = *b->m[mi].pg;
        for (int tid = 0; tid < (int)pg.tensors.size(); ++tid)
            if (pg.tensors[tid].is_const_one) ones.push_back({tensor_ptr(mi, tid)});
    }
    // final tasks and their slot tables
    b->h_final.clear();
    struct Tbl { size_t sx, zz, sxd, zzd, sz, sy; };
    std::vector<Tbl> tbl;   // offsets in ints
    for (int mi = 0; mi < (int)b->m.size(); ++mi) {
        const Member& mb = b->m[mi];
        const Program& pg = *mb.pg;
        Tbl tb;
        tb.sx = ints.size();
        for (int s : pg.sx_slot) ints.push_back((int)(mb.slot_base + s));
        tb.zz = ints.size();
        for (int s : pg.zz_slot) ints.push_back((int)(mb.slot_base + s));
        tb.sxd = ints.size();
        for (int s : pg.sx_den) ints.push_back((int)(mb.slot_base + s));
        tb.zzd = ints.size();
        for (int s : pg.zz_den) ints.push_back((int)(mb.slot_base + s));
        tb.sz = ints.size();
        for (int s : pg.sz_slot) ints.push_back((int)(mb.slot_base + s));
        tb.sy = ints.size();
        for (int s : pg.sy_slot) ints.push_back((int)(mb.slot_base + s));
        tbl.push_back(tb);
    }
    lay.task_bytes = tasks.size();
    lay.status_off = up(lay.tasks_off + tasks.size());
    lay.final_off = up(lay.status_off + sizeof(int));
    lay.ints_off = up(lay.final_off + b->m.size() * sizeof(FinalTask));
    lay.ones_off = up(lay.ints_off + ints.size() * sizeof(int));
    lay.total = up(lay.ones_off + ones.size() * sizeof(ConstOne));
    lay.nones = (int64_t)ones.size();
    lay.nints = (int64_t)ints.size();
    for (int mi = 0; mi < (int)b->m.size(); ++mi) {
        const Member& mb = b->m[mi];
        FinalTask f{};
        f.norm_slot = (int)(mb.slot_base + mb.pg->norm_slot);
        f.n_sites = (int)mb.pg->sx_slot.size();
        f.n_bonds = (int)mb.pg->zz_slot.size();
        f.n_sy = (int)mb.pg->sy_slot.size();
        if (base) {
            const int* ib = reinterpret_cast<const int*>(base + lay.ints_off);
            f.sx_slots = ib + tbl[mi].sx;
            f.zz_slots = ib + tbl[mi].zz;
            f.sx_den = ib + tbl[mi].sxd;
            f.zz_den = ib + tbl[mi].zzd;
            f.sz_slots = ib + tbl[mi].sz;
            f.sy_slots = ib + tbl[mi].sy;
            f.out = reinterpret_cast<double*>(base + lay.res_off) + mb.res_off;
        }
        f.J = 1.0;
        f.h = 0.0;
        b->h_final.push_back(f);
    }
    (void)esize;
    if (tasks_out) tasks_out->swap(tasks);
    if (ints_out) ints_out->swap(ints);
    if (ones_out) ones_out->swap(ones);
}

}  // namespace

std::shared_ptr<const Program> program_cached(int L, int W, int D, tn_schedule sched, tn_precision prec,
                                              tn_work work, int knobs_code, bool cplx) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int, int, int, int>, std::shared_ptr<const Program>> cache;
    // the tuning table's choice for this shape unless the caller names one
    if (knobs_code < 0) knobs_code = tuned_knobs(L, W, D, prec, work).code();
    const auto key = std::make_tuple(L, W, D, (int)sched, (int)prec, (int)work, knobs_code, (int)cplx);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    auto pg = program_build(L, W, D, sched, prec, work, Knobs::from_code(knobs_code), cplx);
    std::lock_guard<std::mutex> g(mu);
    return cache.emplace(key, pg).first->second;
}

tn_status batch_create(tn_ctx* ctx, int n, const int* L, const int* W, const int* D,
                       tn_precision prec, tn_schedule sched, tn_work work, bool alloc,
                       tn_batch** out, size_t* bytes, const BatchOpts* opts) {
    const BatchOpts defaults;
    if (!opts) opts = &defaults;
    if (n <= 0 || !L || !W || !D) { set_error("empty batch"); return TN_ERR_INVALID; }
    if (prec < TN_FP64 || prec > TN_BF16X6 || sched < TN_SCHED_AUTO || sched > TN_SCHED_QUADRANT ||
        !work_valid(work)) {
        set_error("bad enum"); return TN_ERR_INVALID;
    }
    for (int k = 0; k < n; ++k)
        if (L[k] < 1 || L[k] > 16 || W[k] < 1 || W[k] > 16 || D[k] < 1 || D[k] > 4) {
            set_error("lattice size out of range (1..16 x 1..16, D 1..4)");
            return TN_ERR_INVALID;
        }
    auto b = std::make_unique<tn_batch>();
    b->ctx = ctx;
    b->dt = prec == TN_FP64 ? 0 : 1;
    b->work = work;
    b->sched = sched;
    // programs are shared between members (and batches) of the same shape
    for (int k = 0; k < n; ++k) {
        std::shared_ptr<const Program> pg;
        try {
            pg = opts->program ? opts->program
                               : program_cached(L[k], W[k], D[k], sched, prec, work,
                                                (int)opts->member_knobs.size() == n ? opts->member_knobs[k]
                                                                                     : opts->knobs,
                                                opts->complex_sites);
            if (pg->plan.L != L[k] || pg->plan.W != W[k] || pg->plan.D != D[k] || pg->cplx != opts->complex_sites) {
                set_error("the given program is for another lattice shape");
                return TN_ERR_INVALID;
            }
        } catch (const std::exception& e) {
            set_error(e.what());
            return TN_ERR_INVALID;
        }
        Member mb;
        mb.pg = pg;
        mb.L = L[k]; mb.W = W[k]; mb.D = D[k];
        b->m.push_back(mb);
    }
    b->arena_external = opts->arena_external;
    materialize(b.get(), nullptr, nullptr, nullptr, nullptr);
    if (alloc && b->arena_external && (!opts->ext_arena || opts->ext_arena_bytes < b->arena_bytes)) {
        set_error("the shared arena is smaller than the batch's tensors");
        return TN_ERR_INVALID;
    }
    b->ext_arena = opts->ext_arena;
    if (bytes) *bytes = b->lay.total;
    if (!alloc) { *out = b.release(); return TN_OK; }
    if (!ctx || ctx->device < 0) { set_error("context has no device"); return TN_ERR_NO_DEVICE; }
    const size_t need = b->lay.total;
    size_t cur = ctx->used.load();
    do {
        if (cur + need > ctx->budget) {
            set_error("footprint " + std::to_string(need) + " B exceeds the remaining budget");
            return TN_ERR_OVER_BUDGET;
        }
    } while (!ctx->used.compare_exchange_weak(cur, cur + need));
    cudaSetDevice(ctx->device);
    b->stream = opts->stream ? opts->stream : ctx->stream;
    b->async_alloc = opts->async_alloc;
    b->use_graph = opts->use_graph;
    cudaError_t e = b->async_alloc ? cudaMallocAsync(reinterpret_cast<void**>(&b->buf), need, b->stream)
                                   : cudaMalloc(&b->buf, need);
    if (e != cudaSuccess) {
        b->buf = nullptr;
        ctx->used -= need;
        return cuda_status(e, "device allocation");
    }
    std::vector<int> ints;
    std::vector<ConstOne> ones;
    materialize(b.get(), b->buf, &b->h_tasks, &ints, &ones);
    b->h_ints.swap(ints);
    b->h_ones.swap(ones);
    // stream-ordered uploads; the host copies live in the batch until it is destroyed
    e = cudaMemcpyAsync(b->buf + b->lay.tasks_off, b->h_tasks.data(), b->h_tasks.size(), cudaMemcpyHostToDevice,
                        b->stream);
    if (e == cudaSuccess && !b->h_ints.empty())
        e = cudaMemcpyAsync(b->buf + b->lay.ints_off, b->h_ints.data(), b->h_ints.size() * sizeof(int),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !b->h_ones.empty())
        e = cudaMemcpyAsync(b->buf + b->lay.ones_off, b->h_ones.data(), b->h_ones.size() * sizeof(ConstOne),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->buf + b->lay.in_off, 0, (size_t)b->lay.nin * 8, b->stream);
    if (e == cudaSuccess && !b->async_alloc) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        if (b->async_alloc) cudaFreeAsync(b->buf, b->stream); else cudaFree(b->buf);
        b->buf = nullptr;
        ctx->used -= need;
        return cuda_status(e, "batch upload");
    }
    b->h_h.assign(b->m.size(), 0.0);
    *out = b.release();
    return TN_OK;
}

void batch_destroy(tn_batch* b) {
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->buf) {
        if (b->async_alloc) cudaFreeAsync(b->buf, b->stream);
        else cudaFree(b->buf);
        b->ctx->used -= b->lay.total;
    }
    delete b;
}

namespace {

cudaError_t issue(tn_batch* b, cudaStream_t st, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* ev) {
    char* base = b->buf;
    Slot* slots = reinterpret_cast<Slot*>(base + b->lay.slots_off);
    int* status = reinterpret_cast<int*>(base + b->lay.status_off);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    e = launch_init(slots, b->lay.nslots, reinterpret_cast<const ConstOne*>(base + b->lay.ones_off),
                    (int)b->lay.nones, b->dt, st);
    if (e != cudaSuccess) return e;
    const char* tb = base + b->lay.tasks_off;
    for (size_t li = 0; li < b->launches.size(); ++li) {
        const Launch& L = b->launches[li];
        if (ev) cudaEventRecord((*ev)[li].first, st);
        const void* tp = tb + L.task_off;
        const int* tmap = L.map_off ? reinterpret_cast<const int*>(tb + L.map_off) : nullptr;
        switch (L.kind) {
            case OP_SITEMAT:
                e = launch_sitemat(L.dt, static_cast<const SiteMatTask*>(tp), L.ntasks, slots, st);
                break;
            case OP_ABSORB:
            case OP_ABSORB_DOT:
                if (L.variant >= 3 && L.variant < 10)
                    e = launch_tc_absorb(L.variant - 1, L.kind == OP_ABSORB_DOT, static_cast<const AbsorbTask*>(tp),
                                         L.ntasks, L.nblocks, slots, status, st);
                else
                    e = launch_absorb(L.dt, L.kind == OP_ABSORB_DOT, L.K, L.N, static_cast<const AbsorbTask*>(tp),
                                      L.ntasks, L.nblocks, slots, st, L.variant, tmap);
                break;
            case OP_GEMM:
            case OP_GEMM_DOT:
                e = launch_gemm(L.dt, L.kind == OP_GEMM_DOT, static_cast<const GemmTask*>(tp), L.ntasks,
                                L.nblocks, slots, st, L.variant);
                break;
            case OP_ABSORB2:
            case OP_ABSORB2_DOT:
                e = launch_absorb2(L.kind == OP_ABSORB2_DOT, L.K, L.N, static_cast<const AbsorbTask*>(tp), L.ntasks,
                                   L.nblocks, slots, st, tmap);
                break;
            case OP_DOT:
                e = launch_dot(L.dt, static_cast<const DotTask*>(tp), L.ntasks, L.nblocks, slots, st, tmap);
                break;
            case OP_TC_SPLIT:
                e = launch_tc_split(static_cast<const TcSplitTask*>(tp), L.ntasks, L.nblocks, slots, st);
                break;
            case OP_TC_GEMM:
                e = launch_tc_gemm((L.variant % 10000) / 1000, false, L.variant % 1000,
                                   static_cast<const TcGemmTask*>(tp), L.ntasks, L.nblocks, slots, status, st,
                                   L.variant >= 10000);
                break;
            case OP_TC_GEMM_DOT:
                e = launch_tc_gemm_dot((L.variant % 10000) / 1000, L.variant % 1000,
                                       static_cast<const TcGemmTask*>(tp), L.ntasks, L.nblocks, slots, status, st);
                break;
        }
        if (ev) cudaEventRecord((*ev)[li].second, st);
        if (e != cudaSuccess) return e;
    }
    return launch_final(reinterpret_cast<const FinalTask*>(base + b->lay.final_off), (int)b->m.size(), slots, st);
}

}  // namespace

tn_status batch_run_plain(tn_batch* b, cudaStream_t st);

namespace {
// Host-side fault injection: mark this run's status word as if a bounded
// device wait had run out (no kernel is disturbed; tn_ctx_inject_wait_timeout).
tn_status inject_after_run(tn_batch* b, cudaStream_t st, tn_status s) {
    tn_ctx* ctx = b->ctx;
    if (s != TN_OK) return s;
    int v = ctx->inject_timeouts.load();
    while (v > 0 && !ctx->inject_timeouts.compare_exchange_weak(v, v - 1)) {
    }
    if (v <= 0) return s;
    return cuda_status(cudaMemsetAsync(b->buf + b->lay.status_off, 1, 1, st), "injected status");
}
}  // namespace

tn_status batch_run(tn_batch* b, cudaStream_t st) {
    return inject_after_run(b, st, batch_run_plain(b, st));
}

tn_status batch_run_plain(tn_batch* b, cudaStream_t st) {
    tn_ctx* ctx = b->ctx;
    cudaSetDevice(ctx->device);
    // the fields of the final step (J, h) change between runs: refresh them
    cudaError_t e = cudaMemcpyAsync(b->buf + b->lay.final_off, b->h_final.data(),
                                    b->h_final.size() * sizeof(FinalTask), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "final table upload");
    if (ctx->profiling) {
        std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev(b->launches.size());
        for (auto& p : ev) { cudaEventCreate(&p.first); cudaEventCreate(&p.second); }
        e = issue(b, st, &ev);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            std::lock_guard<std::mutex> g(ctx->mu);
            for (size_t li = 0; li < b->launches.size(); ++li) {
                float ms = 0;
                cudaEventElapsedTime(&ms, ev[li].first, ev[li].second);
                KStat& s = ctx->stats[family_of(b->launches[li].kind)];
                s.launches += 1;
                s.ms += ms;
                s.bytes += b->launches[li].bytes;
                s.macs += b->launches[li].macs;
            }
        }
        for (auto& p : ev) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
        return cuda_status(e, "profiled run");
    }
    if (!b->use_graph) return cuda_status(issue(b, st, nullptr), "batch run");
    if (!b->gexec) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status(e, "begin capture");
        cudaError_t ei = issue(b, st, nullptr);
        e = cudaStreamEndCapture(st, &g);
        if (ei != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_status(ei, "capture issue"); }
        if (e != cudaSuccess) return cuda_status(e, "end capture");
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { b->gexec = nullptr; return cuda_status(e, "graph instantiate"); }
    }
    return cuda_status(cudaGraphLaunch(b->gexec, st), "graph launch");
}

cudaError_t batch_issue(tn_batch* b, cudaStream_t st) { return issue(b, st, nullptr); }

}  // namespace tn
