// Program builder: turns a plan (planner.cpp) into the list of pairwise
// contractions that yield the norm and, for TN_WORK_ENERGY, every <X_k>,
// every <Z_k> and every nearest-neighbour <Z_i Z_j> (Sec. 5 contracts the
// network once more for every site and every pair); the bond work kinds give
// <A_i B_j> on every bond for A, B in {X, Z} instead.
//
// Structure (oriented lattice, corners TL, TR, BL, BR):
//   F[q][t]   forward chain of corner q: F[q][t] = absorb(F[q][t-1], E_I(site t))
//   M_top = TL TR^T, M_bot = BL BR^T, norm = <M_top, M_bot>     (ring closure)
//   Env[TL] = M_bot TR, Env[TR] = M_bot^T TL, Env[BL] = M_top BR, Env[BR] = M_top^T BL
//   G[q][t]   environment sweep: G[q][T] = Env[q],
//             G[q][t-1] = absorb(G[q][t], E_I(site t)^T), so <F[q][t], G[q][t]> = norm
//   site k at step t:      <absorb(F[q][t-1], E_O), G[q][t]> for O = X, Z and
//                          I (the local norm) in one pass where the FP32
//                          kernel serves the step
//   bond inside corner q:  Z inserted at the first site, the chain carried to
//                          the second site (1 step, or one frame row), Z there,
//                          dotted with G at that step; consecutive steps of one
//                          frame row fused in pairs
//   bond across a cut:     both corners regrown with Z to their last step, then
//                          one dense product with the rest of the ring.
// Every value is exact (no truncation); reusing the unchanged corners and
// environments instead of one full contraction per observable changes only the
// amount of work.  Every tensor is a separate SSA value; an interval allocator
// packs their lifetimes (wave of production .. last wave that reads them) into
// one arena.
#include <algorithm>
#include <cstring>
#include <functional>
#include <map>
#include <stdexcept>

#include "tn_internal.h"
#include "tn_kernels.h"

namespace tn {

namespace {

struct SiteRef {
    int q = -1, t = -1, k = -1, c = -1;   // corner, 1-based chain step, frame row / column
};

class Builder {
public:
    Builder(Program& pg) : pg_(pg) {}

    int tensor(int64_t n, int level) {
        Tensor t;
        t.n = n;
        t.level = level;
        t.slot = pg_.n_slots++;
        pg_.tensors.push_back(t);
        return (int)pg_.tensors.size() - 1;
    }
    int scalar(int level) { return tensor(0, level); }
    int const_one() {
        if (one_ < 0) {
            one_ = tensor(1, 0);
            pg_.tensors[one_].is_const_one = true;
        }
        return one_;
    }
    void use(int tid, int level) {
        Tensor& t = pg_.tensors[tid];
        t.last_use = std::max(t.last_use, level);
    }
    int level_of(int tid) const { return pg_.tensors[tid].level; }

    int add(Op op) {
        max_level_ = std::max(max_level_, op.level);
        pg_.ops.push_back(op);
        return (int)pg_.ops.size() - 1;
    }
    // the last wave any op so far runs in
    int max_level() const { return max_level_; }
    // Every op created while a global floor is set starts after that wave
    // (the recompute form's stages: each stage starts when the previous one
    // has finished, so the arena reuses the previous stage's memory).
    void set_gfloor(int f) { gfloor_ = f; }

    // Site matrix of `site` with physical operator `phys` in its corner's frame.
    int sitemat(int site, int phys, const CornerPlan& cp, const Step& s) {
        auto key = std::make_pair(site, phys);
        auto it = E_.find(key);
        if (it != E_.end()) return it->second;
        // interior D = 3 steps: keep the two layer factors (Sec. 5, bra and
        // ket layers) and absorb them one after the other; without that choice
        // the double-layer matrix is formed (and, in the split-BF16 precisions,
        // the step runs on the tensor cores)
        const bool factored = s.K == 81 && s.N == 81 && pg_.knobs.factor_d3;
        const int e = tensor(factored ? (int64_t)kFactorEntries : (int64_t)s.K * s.N, 0);
        pg_.tensors[e].factored = factored;
        Op op;
        op.kind = OP_SITEMAT;
        op.level = 0;
        op.out = e;
        op.factored = factored;
        op.site = site;
        op.phys = phys;
        op.K = s.K;
        op.N = s.N;
        std::memcpy(op.map, cp.map, sizeof(op.map));
        for (int k = 0; k < 4; ++k) op.fdim[k] = pg_.site_dims[4 * site + cp.map[k]];
        // the chain step's leg groups must be the site's frame legs (double layer)
        const int fu = op.fdim[0], fl = op.fdim[1], fd = op.fdim[2], fr = op.fdim[3];
        if (s.K != fl * fl * fu * fu || s.N != fd * fd * fr * fr)
            throw std::logic_error("site matrix shape does not match its chain step");
        op.bytes = (double)pg_.tensors[e].n * pg_.esize;
        add(op);
        E_[key] = e;
        return e;
    }

    // out = absorb(in, E) with the shape of step s (transposed: backward sweep).
    // Ops created while a floor is set start no earlier than that wave (used to
    // run observable chains in memory-bounded stages).
    void set_floor(int f) { floor_ = f; }

    int absorb(int in, int E, const Step& s, bool trans) {
        const int level = std::max({level_of(in), level_of(E), floor_, gfloor_}) + 1;
        const int64_t nout = trans ? s.n_in : s.n_out;
        const int out = tensor(nout, level);
        Op op;
        op.kind = OP_ABSORB;
        op.level = level;
        op.in = in; op.E = E; op.out = out;
        op.P = s.P; op.S = s.S;
        op.K = trans ? s.N : s.K;
        op.N = trans ? s.K : s.N;
        op.transE = trans;
        op.factored = pg_.tensors[E].factored;
        // wide double-layer steps (D = 3 interior, K = N = 81) not in the
        // factored form go to the tensor cores
        if (pg_.nsplit && op.K == 81 && op.N == 81 && !op.factored) op.nsplit = pg_.nsplit;
        op.bytes = (double)(s.n_in + s.n_out) * pg_.esize;
        // the factored form does 2 x 2 x 9^3 multiply-adds per outer position instead of 81^2
        op.macs = op.factored ? (double)s.P * s.S * 2916.0 : (double)s.mac;
        use(in, level); use(E, level);
        add(op);
        return out;
    }

    // scalar = <absorb(in, E), adj> with the shape of step s.
    int absorb_dot(int in, int E, int adj, const Step& s) {
        const int level = std::max({level_of(in), level_of(E), level_of(adj), gfloor_}) + 1;
        const int out = scalar(level);
        Op op;
        op.kind = OP_ABSORB_DOT;
        op.level = level;
        op.in = in; op.E = E; op.adj = adj; op.out = out;
        op.P = s.P; op.S = s.S; op.K = s.K; op.N = s.N;
        op.factored = pg_.tensors[E].factored;
        if (pg_.nsplit && op.K == 81 && op.N == 81 && !op.factored) op.nsplit = pg_.nsplit;
        op.bytes = (double)(s.n_in + s.n_out) * pg_.esize;
        op.macs = (op.factored ? (double)s.P * s.S * 2916.0 : (double)s.mac) + (double)s.n_out;
        use(in, level); use(E, level); use(adj, level);
        add(op);
        return out;
    }

    // Whether two consecutive steps of one frame row can run fused (FP32, D = 2:
    // the first step 4 or 16 -> (dn, h') = 4 x 4, the second (h', u) = 4 x 4 ->
    // N2, at least 8 trailing positions so every warp access covers whole sectors).
    bool pair_ok(const Step& a, const Step& b) const {
        if (!pg_.knobs.fuse_pairs) return false;
        if (pg_.dt != DT_F32 || a.corner != b.corner || a.k != b.k || b.c != a.c + 1) return false;
        if (!(a.K == 4 || a.K == 16) || a.N != 16 || b.K != 16 || !(b.N == 1 || b.N == 4 || b.N == 16)) return false;
        return b.P == 4 * a.P && a.S == 4 * b.S && b.S >= 8;
    }

    // absorb(absorb(in, E1), E2) for the consecutive steps a, b (pair_ok).
    int absorb2(int in, int E1, int E2, const Step& a, const Step& b) {
        const int level = std::max({level_of(in), level_of(E1), level_of(E2), floor_, gfloor_}) + 1;
        const int out = tensor(b.n_out, level);
        Op op;
        op.kind = OP_ABSORB2;
        op.level = level;
        op.in = in; op.E = E1; op.E2 = E2; op.out = out;
        op.P = a.P; op.S = b.S; op.K = a.K; op.N = b.N;
        op.bytes = (double)(a.n_in + b.n_out) * pg_.esize;
        op.macs = (double)a.mac + (double)b.mac;
        use(in, level); use(E1, level); use(E2, level);
        add(op);
        return out;
    }

    // <absorb(absorb(in, E1), E2), adj> for the consecutive steps a, b (pair_ok).
    int absorb2_dot(int in, int E1, int E2, int adj, const Step& a, const Step& b) {
        const int level =
            std::max({level_of(in), level_of(E1), level_of(E2), level_of(adj), floor_, gfloor_}) + 1;
        const int out = scalar(level);
        Op op;
        op.kind = OP_ABSORB2_DOT;
        op.level = level;
        op.in = in; op.E = E1; op.E2 = E2; op.adj = adj; op.out = out;
        op.P = a.P; op.S = b.S; op.K = a.K; op.N = b.N;
        op.bytes = (double)(a.n_in + b.n_out) * pg_.esize;
        op.macs = (double)a.mac + (double)b.mac + (double)b.n_out;
        use(in, level); use(E1, level); use(E2, level); use(adj, level);
        add(op);
        return out;
    }

    // Whether the FP32 streaming absorption serves this step (it has the triple dot).
    bool dual_ok(const Step& s) const {
        if (!pg_.knobs.site_triple) return false;
        const int v = absorb_variant(pg_.dt == DT_F64 ? 0 : 1, s.P, s.S, s.K, s.N);
        return pg_.dt == DT_F32 && !(pg_.nsplit && s.K == 81 && s.N == 81) && (v == 1 || v == 2);
    }

    // (<absorb(in, E), adj>, <absorb(in, E2), adj>, <absorb(in, E3), adj>) in
    // one pass over in and adj.
    std::tuple<int, int, int> absorb_dot3(int in, int E, int E2, int E3, int adj, const Step& s) {
        const int level =
            std::max({level_of(in), level_of(E), level_of(E2), level_of(E3), level_of(adj), gfloor_}) + 1;
        const int out = scalar(level), out2 = scalar(level), out3 = scalar(level);
        Op op;
        op.kind = OP_ABSORB_DOT;
        op.level = level;
        op.in = in; op.E = E; op.E2 = E2; op.E3 = E3; op.adj = adj;
        op.out = out; op.out2 = out2; op.out3 = out3;
        op.P = s.P; op.S = s.S; op.K = s.K; op.N = s.N;
        op.bytes = (double)(s.n_in + s.n_out) * pg_.esize;
        op.macs = 3.0 * ((double)s.mac + (double)s.n_out);
        use(in, level); use(E, level); use(E2, level); use(E3, level); use(adj, level);
        add(op);
        return {out, out2, out3};
    }

    // Tiled BF16 planes of the operand X[r][k] = src[r*sr + k*sk] (one per view).
    int tc_split(int src, int64_t R, int64_t Kd, int64_t sr, int64_t sk) {
        // the recompute form splits per product, so no plane set outlives its product
        auto key = std::make_tuple(src, R, Kd, sr, sk);
        auto it = split_.find(key);
        if (it != split_.end() && !pg_.knobs.recompute) return it->second;
        const int64_t Rp = (R + kTcRowPad - 1) / kTcRowPad * kTcRowPad, Kp = (Kd + 63) / 64 * 64;
        const int level = std::max(level_of(src), gfloor_) + 1;
        // BF16 planes counted in 4-byte units of the FP32 arena
        const int out = tensor((int64_t)pg_.nsplit * Rp * Kp / 2, level);
        Op op;
        op.kind = OP_TC_SPLIT;
        op.level = level;
        op.A = src; op.out = out;
        op.gm = R; op.gk = Kd; op.sam = sr; op.sak = sk;
        op.Rp = Rp; op.Kp = Kp; op.nsplit = pg_.nsplit;
        op.bytes = (double)R * Kd * 4 + (double)pg_.nsplit * Rp * Kp * 2;
        use(src, level);
        add(op);
        split_[key] = out;
        return out;
    }

    // C[m][n] = sum_k A(m,k) B(k,n); dot partner Cd -> scalar.
    int gemm(int A, int B, int64_t M, int64_t N, int64_t K, int64_t sam, int64_t sak,
             int64_t sbk, int64_t sbn, int Cd = -1) {
        // tensor cores for products of at least 2^26 multiply-adds: below that
        // (e.g. the 256^3 ring of an 8 x 8 D = 2 lattice: 14.2 against 12.0 ms
        // per batch of 256 lattices in BF16x6) splitting the operands and the
        // per-tile set-up cost more than the FP32 SIMT product
        if (pg_.nsplit && pg_.knobs.tc_products && M >= 128 && N >= 128 && K >= 64 &&
            (M * N * K >= (1LL << 26) || pg_.knobs.tc_small)) {
            // tensor cores: C = A' B'^T with A'[m][k] = A(m,k) and B'[n][k] = B(k,n)
            const int Ap = tc_split(A, M, K, sam, sak);
            const int Bp = tc_split(B, N, K, sbn, sbk);
            int lv = std::max({level_of(Ap), level_of(Bp), gfloor_}) + 1;
            if (Cd >= 0) lv = std::max(lv, level_of(Cd) + 1);
            const int o = Cd >= 0 ? scalar(lv) : tensor(M * N, lv);
            Op op;
            op.kind = Cd >= 0 ? OP_TC_GEMM_DOT : OP_TC_GEMM;
            op.level = lv;
            op.A = Ap; op.B = Bp; op.C = Cd; op.out = o;
            op.A_src = A; op.B_src = B;
            op.gm = M; op.gn = N; op.gk = K;
            op.Kp = (K + 63) / 64 * 64;
            op.nsplit = pg_.nsplit;
            op.bytes = (double)pg_.nsplit * ((M + kTcRowPad - 1) / kTcRowPad + (N + kTcRowPad - 1) / kTcRowPad) *
                           kTcRowPad * op.Kp * 2 + (double)M * N * 4;
            op.macs = (double)M * N * K;
            use(Ap, lv); use(Bp, lv); use(A, lv); use(B, lv);
            if (Cd >= 0) use(Cd, lv);
            add(op);
            return o;
        }
        int level = std::max({level_of(A), level_of(B), gfloor_}) + 1;
        if (Cd >= 0) level = std::max(level, level_of(Cd) + 1);
        const int out = Cd >= 0 ? scalar(level) : tensor(M * N, level);
        Op op;
        op.kind = Cd >= 0 ? OP_GEMM_DOT : OP_GEMM;
        op.level = level;
        op.A = A; op.B = B; op.C = Cd; op.out = out;
        op.gm = M; op.gn = N; op.gk = K;
        op.sam = sam; op.sak = sak; op.sbk = sbk; op.sbn = sbn;
        op.bytes = (double)(M * K + K * N + M * N) * pg_.esize;
        op.macs = (double)M * N * K;
        use(A, level); use(B, level);
        if (Cd >= 0) use(Cd, level);
        add(op);
        return out;
    }

    int dot(int A, int B, int64_t n) {
        const int level = std::max({level_of(A), level_of(B), gfloor_}) + 1;
        const int out = scalar(level);
        Op op;
        op.kind = OP_DOT;
        op.level = level;
        op.A = A; op.B = B; op.out = out;
        op.gm = n;
        op.bytes = 2.0 * n * pg_.esize;
        op.macs = (double)n;
        use(A, level); use(B, level);
        add(op);
        return out;
    }

private:
    Program& pg_;
    int one_ = -1;
    int floor_ = 0;
    int gfloor_ = 0;
    int max_level_ = 0;
    std::map<std::pair<int, int>, int> E_;
    std::map<std::tuple<int, int64_t, int64_t, int64_t, int64_t>, int> split_;
};

// Greedy first-fit interval packing of tensor lifetimes, wave by wave.
int64_t pack_arena(Program& pg) {
    const int64_t align = 256;
    struct Block { int64_t off, len; };
    std::vector<Block> freel;   // sorted by offset
    int64_t top = 0;
    int max_level = 0;
    for (const auto& t : pg.tensors) max_level = std::max({max_level, t.level, t.last_use});
    std::vector<std::vector<int>> born(max_level + 1), dies(max_level + 2);
    for (int k = 0; k < (int)pg.tensors.size(); ++k) {
        Tensor& t = pg.tensors[k];
        if (t.n == 0) continue;
        if (t.last_use < t.level) t.last_use = t.level;
        born[t.level].push_back(k);
        dies[t.last_use + 1].push_back(k);
    }
    auto release = [&](int64_t off, int64_t len) {
        freel.push_back({off, len});
        std::sort(freel.begin(), freel.end(), [](const Block& a, const Block& b) { return a.off < b.off; });
        std::vector<Block> merged;
        for (const auto& b : freel) {
            if (!merged.empty() && merged.back().off + merged.back().len == b.off) merged.back().len += b.len;
            else merged.push_back(b);
        }
        freel.swap(merged);
        if (!freel.empty() && freel.back().off + freel.back().len == top) {
            top = freel.back().off;
            freel.pop_back();
        }
    };
    int64_t high = 0;
    for (int lv = 0; lv <= max_level; ++lv) {
        for (int k : dies[lv]) {
            const Tensor& t = pg.tensors[k];
            release(t.offset, (t.n * pg.esize + align - 1) / align * align);
        }
        for (int k : born[lv]) {
            Tensor& t = pg.tensors[k];
            const int64_t len = (t.n * pg.esize + align - 1) / align * align;
            bool placed = false;
            for (size_t b = 0; b < freel.size(); ++b) {
                if (freel[b].len >= len) {
                    t.offset = freel[b].off;
                    freel[b].off += len;
                    freel[b].len -= len;
                    if (freel[b].len == 0) freel.erase(freel.begin() + b);
                    placed = true;
                    break;
                }
            }
            if (!placed) {
                t.offset = top;
                top += len;
            }
            high = std::max(high, top);
        }
    }
    return high;
}

}  // namespace

std::shared_ptr<const Program> program_build(int L, int W, int D, tn_schedule sched,
                                             tn_precision prec, tn_work work, Knobs knobs, bool cplx) {
    return program_build_plan(plan_choose(L, W, D, sched, work), prec, work, knobs, nullptr, cplx);
}

std::shared_ptr<const Program> program_build_plan(const Plan& plan, tn_precision prec, tn_work work, Knobs knobs,
                                                  const std::vector<PairSpec>* pairs, bool cplx) {
    auto pgp = std::make_shared<Program>();
    Program& pg = *pgp;
    pg.plan = plan;
    pg.cplx = cplx;
    // the two-pass absorption keeps the double layer as bra x ket factors; the
    // real basis of complex site matrices mixes the two layers, so it is off
    if (cplx) knobs.factor_d3 = false;
    pg.knobs = knobs;
    const int L = plan.L, W = plan.W, D = plan.D;
    pg.work = work;
    pg.dt = prec == TN_FP64 ? DT_F64 : DT_F32;
    pg.nsplit = prec == TN_BF16X3 ? 2 : (prec == TN_BF16X6 ? 3 : 0);
    pg.esize = pg.dt == DT_F64 ? 8 : 4;
    const Plan& pl = pg.plan;
    const int nsite = L * W;

    // raw FP64 input layout, [p][u][l][dn][rt] per site, row-major sites
    // (complex: the site's real parts, then its imaginary parts)
    pg.site_offset.resize(nsite + 1);
    pg.site_dims.resize(4 * nsite);
    pg.site_offset[0] = 0;
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < W; ++c) {
            const int s = r * W + c;
            int* dm = &pg.site_dims[4 * s];
            dm[0] = r == 0 ? 1 : D;
            dm[1] = c == 0 ? 1 : D;
            dm[2] = r == L - 1 ? 1 : D;
            dm[3] = c == W - 1 ? 1 : D;
            pg.site_offset[s + 1] = pg.site_offset[s] + (cplx ? 4LL : 2LL) * dm[0] * dm[1] * dm[2] * dm[3];
        }
    pg.input_bytes = pg.site_offset[nsite] * 8;

    Builder bd(pg);
    std::vector<SiteRef> where(nsite);
    for (int q = 0; q < 4; ++q) {
        const auto& st = pl.corner[q].steps;
        for (int t = 0; t < (int)st.size(); ++t) {
            SiteRef& w = where[st[t].r * W + st[t].col];
            w.q = q; w.t = t + 1; w.k = st[t].k; w.c = st[t].c;
        }
    }
    auto step_of = [&](int q, int t) -> const Step& { return pl.corner[q].steps[t - 1]; };
    auto site_of = [&](int q, int t) { const Step& s = step_of(q, t); return s.r * W + s.col; };
    auto E_at = [&](int q, int t, int phys) {
        return bd.sitemat(site_of(q, t), phys, pl.corner[q], step_of(q, t));
    };

    // forward chains
    std::vector<int> F[4];
    int Qt[4];
    for (int q = 0; q < 4; ++q) {
        const int T = (int)pl.corner[q].steps.size();
        F[q].assign(T + 1, -1);
        F[q][0] = bd.const_one();
        for (int t = 1; t <= T; ++t) F[q][t] = bd.absorb(F[q][t - 1], E_at(q, t, PH_I), step_of(q, t), false);
        Qt[q] = F[q][T];
    }
    const int64_t hbL = pl.hb_L, hbR = pl.hb_R, vrT = pl.vr_T, vrB = pl.vr_B;
    // ring closure
    const int Mtop = bd.gemm(Qt[TL], Qt[TR], hbL, hbR, vrT, vrT, 1, 1, vrT);
    const int Mbot = bd.gemm(Qt[BL], Qt[BR], hbL, hbR, vrB, vrB, 1, 1, vrB);
    pg.norm_slot = pg.tensors[bd.dot(Mtop, Mbot, hbL * hbR)].slot;

    if (work != TN_WORK_NORM) {
        // energies: every site and the ZZ bonds; bond work kinds: the bonds
        // alone with operators A on each bond's first site and B on its second
        const bool with_sites = work == TN_WORK_ENERGY && !pairs;
        const int bondA = work_is_bonds(work) ? work_bond_a(work) : PH_Z;
        const int bondB = work_is_bonds(work) ? work_bond_b(work) : PH_Z;
        const bool recompute = pg.knobs.recompute;
        auto nonempty = [&](int q) { return !pl.corner[q].steps.empty(); };
        // the rest of the ring seen from corner q
        auto env_of = [&](int q) {
            switch (q) {
                case TL: return bd.gemm(Mbot, Qt[TR], hbL, vrT, hbR, hbR, 1, vrT, 1);
                case TR: return bd.gemm(Mbot, Qt[TL], hbR, vrT, hbL, 1, hbR, vrT, 1);
                case BL: return bd.gemm(Mtop, Qt[BR], hbL, vrB, hbR, hbR, 1, vrB, 1);
                default: return bd.gemm(Mtop, Qt[BL], hbR, vrB, hbL, 1, hbR, vrB, 1);
            }
        };
        // environment sweeps (cached form)
        std::vector<int> G[4];
        if (!recompute) {
            int Env[4] = {-1, -1, -1, -1};
            for (int q = 0; q < 4; ++q)
                if (nonempty(q)) Env[q] = env_of(q);
            for (int q = 0; q < 4; ++q) {
                const int T = (int)pl.corner[q].steps.size();
                G[q].assign(T + 1, -1);
                if (!T) continue;
                G[q][T] = Env[q];
                for (int t = T; t >= 2; --t) G[q][t - 1] = bd.absorb(G[q][t], E_at(q, t, PH_I), step_of(q, t), true);
            }
        }
        // norm along each step's path: <F[q][t], G[q][t]> (from the site's triple
        // absorb-dot where the streaming kernel serves the step, else a dot).
        // Dividing by it cancels the rounding the numerator shares with it;
        // FP64 has no rounding worth cancelling at the library's tolerance, so
        // there every ratio takes the ring's norm and the extra dots and ring
        // products of the path norms are not built.  Fm gives F[q][t-1] (the
        // recompute form takes F[q][t] one step from it).
        const bool path_norms = pg.dt != DT_F64;
        std::map<std::pair<int, int>, int> local_norm;
        auto norm_at = [&](int q, int t, int Gt, const std::function<int()>& Fm) {
            if (!path_norms) return pg.norm_slot;
            auto key = std::make_pair(q, t);
            auto it = local_norm.find(key);
            if (it != local_norm.end()) return it->second;
            const int Ft = recompute ? bd.absorb(Fm(), E_at(q, t, PH_I), step_of(q, t), false) : F[q][t];
            const int v = bd.dot(Ft, Gt, step_of(q, t).n_out);
            const int sl = pg.tensors[v].slot;
            local_norm[key] = sl;
            return sl;
        };
        // one site's observables from F[q][t-1] and G[q][t]
        pg.sx_slot.assign(with_sites ? nsite : 0, -1);
        pg.sz_slot.assign(with_sites ? nsite : 0, -1);
        pg.sx_den.assign(with_sites ? nsite : 0, -1);
        pg.sy_slot.assign(with_sites && cplx ? nsite : 0, -1);
        auto emit_site = [&](int s, int Fm, int Gt) {
            const SiteRef& w = where[s];
            const Step& st = step_of(w.q, w.t);
            if (bd.dual_ok(st)) {
                // the site's <X>, <Z> and the local norm <absorb(F[t-1], E_I), G[t]> in one pass
                const auto v3 = bd.absorb_dot3(Fm, E_at(w.q, w.t, PH_X), E_at(w.q, w.t, PH_Z),
                                               E_at(w.q, w.t, PH_I), Gt, st);
                pg.sx_slot[s] = pg.tensors[std::get<0>(v3)].slot;
                pg.sz_slot[s] = pg.tensors[std::get<1>(v3)].slot;
                local_norm[std::make_pair(w.q, w.t)] = pg.tensors[std::get<2>(v3)].slot;
            } else {
                const int vx = bd.absorb_dot(Fm, E_at(w.q, w.t, PH_X), Gt, st);
                const int vz = bd.absorb_dot(Fm, E_at(w.q, w.t, PH_Z), Gt, st);
                pg.sx_slot[s] = pg.tensors[vx].slot;
                pg.sz_slot[s] = pg.tensors[vz].slot;
            }
            if (cplx) pg.sy_slot[s] = pg.tensors[bd.absorb_dot(Fm, E_at(w.q, w.t, PH_Y), Gt, st)].slot;
            pg.sx_den[s] = norm_at(w.q, w.t, Gt, [&] { return Fm; });
        };
        // bonds, output order: horizontal row-major, then vertical row-major
        // the correlators to form: every nearest-neighbour bond with (A, B), or the caller's pairs
        std::vector<PairSpec> bonds;
        if (pairs) {
            bonds = *pairs;
        } else {
            for (int r = 0; r < L; ++r)
                for (int c = 0; c + 1 < W; ++c) bonds.push_back({r * W + c, r * W + c + 1, bondA, bondB});
            for (int r = 0; r + 1 < L; ++r)
                for (int c = 0; c < W; ++c) bonds.push_back({r * W + c, (r + 1) * W + c, bondA, bondB});
        }
        int Xl = -1, Xr = -1;
        int den_cross[6] = {-1, -1, -1, -1, -1, -1};
        // Chain of corner q over steps t0..t1 from x, operator op0 at step t0
        // and I after; with adj >= 0 the last step is instead an absorb-dot
        // with operator op1 and adj.  Consecutive steps of one frame row run as
        // fused pairs where they can.
        auto chain = [&](int q, int x, int t0, int t1, int adj, int op0, int op1) {
            int u = t0;
            while (u <= t1) {
                const int op_u = u == t0 ? op0 : PH_I;
                const bool last_dot = adj >= 0 && u == t1;
                if (u < t1 && bd.pair_ok(step_of(q, u), step_of(q, u + 1))) {
                    const int op_v = (adj >= 0 && u + 1 == t1) ? op1 : PH_I;
                    if (adj >= 0 && u + 1 == t1)
                        return bd.absorb2_dot(x, E_at(q, u, op_u), E_at(q, u + 1, op_v), adj, step_of(q, u),
                                              step_of(q, u + 1));
                    x = bd.absorb2(x, E_at(q, u, op_u), E_at(q, u + 1, op_v), step_of(q, u), step_of(q, u + 1));
                    u += 2;
                    continue;
                }
                if (last_dot) return bd.absorb_dot(x, E_at(q, u, op1), adj, step_of(q, u));
                x = bd.absorb(x, E_at(q, u, op_u), step_of(q, u), false);
                ++u;
            }
            return x;
        };
        // A pair whose sites lie in two corners: both corners regrown with the
        // operators from F[qa][ta-1] and F[qb][tb-1] to their last step, then
        // the product(s) with the rest of the ring.  Each class of such pairs
        // is normalised by the same fused product on the unmodified corners
        // (the norm through the same path).
        auto emit_cross = [&](size_t bi, int qa, int ta, int opa, int qb, int tb, int opb, int Fa, int Fb) {
            const int Ta = (int)pl.corner[qa].steps.size(), Tb = (int)pl.corner[qb].steps.size();
            const int Za = chain(qa, Fa, ta, Ta, -1, opa, PH_I), Zb = chain(qb, Fb, tb, Tb, -1, opb, PH_I);
            int v = -1;
            if (qa == TL && qb == TR) {
                v = bd.gemm(Mbot, Zb, hbL, vrT, hbR, hbR, 1, vrT, 1, Za);
                if (!path_norms) den_cross[0] = pg.norm_slot;
                if (den_cross[0] < 0)
                    den_cross[0] = pg.tensors[bd.gemm(Mbot, Qt[TR], hbL, vrT, hbR, hbR, 1, vrT, 1, Qt[TL])].slot;
                pg.zz_den[bi] = den_cross[0];
            } else if (qa == BL && qb == BR) {
                v = bd.gemm(Mtop, Zb, hbL, vrB, hbR, hbR, 1, vrB, 1, Za);
                if (!path_norms) den_cross[1] = pg.norm_slot;
                if (den_cross[1] < 0)
                    den_cross[1] = pg.tensors[bd.gemm(Mtop, Qt[BR], hbL, vrB, hbR, hbR, 1, vrB, 1, Qt[BL])].slot;
                pg.zz_den[bi] = den_cross[1];
            } else if (qa == TL && qb == BL) {
                if (Xr < 0) Xr = bd.gemm(Qt[TR], Qt[BR], vrT, vrB, hbR, 1, vrT, vrB, 1);
                v = bd.gemm(Za, Zb, vrT, vrB, hbL, 1, vrT, vrB, 1, Xr);
                if (!path_norms) den_cross[2] = pg.norm_slot;
                if (den_cross[2] < 0)
                    den_cross[2] = pg.tensors[bd.gemm(Qt[TL], Qt[BL], vrT, vrB, hbL, 1, vrT, vrB, 1, Xr)].slot;
                pg.zz_den[bi] = den_cross[2];
            } else if (qa == TR && qb == BR) {
                if (Xl < 0) Xl = bd.gemm(Qt[TL], Qt[BL], vrT, vrB, hbL, 1, vrT, vrB, 1);
                v = bd.gemm(Za, Zb, vrT, vrB, hbR, 1, vrT, vrB, 1, Xl);
                if (!path_norms) den_cross[3] = pg.norm_slot;
                if (den_cross[3] < 0)
                    den_cross[3] = pg.tensors[bd.gemm(Qt[TR], Qt[BR], vrT, vrB, hbR, 1, vrT, vrB, 1, Xl)].slot;
                pg.zz_den[bi] = den_cross[3];
            } else if (qa == TL && qb == BR) {
                // diagonal corners: <Za TR^T, BL Zb^T>, two products
                const int P1 = bd.gemm(Za, Qt[TR], hbL, hbR, vrT, vrT, 1, 1, vrT);
                v = bd.gemm(Qt[BL], Zb, hbL, hbR, vrB, vrB, 1, 1, vrB, P1);
                if (!path_norms) den_cross[4] = pg.norm_slot;
                if (den_cross[4] < 0)
                    den_cross[4] = pg.tensors[bd.gemm(Qt[BL], Qt[BR], hbL, hbR, vrB, vrB, 1, 1, vrB, Mtop)].slot;
                pg.zz_den[bi] = den_cross[4];
            } else if (qa == TR && qb == BL) {
                // diagonal corners: <TL Za^T, Zb BR^T>, two products
                const int P1 = bd.gemm(Qt[TL], Za, hbL, hbR, vrT, vrT, 1, 1, vrT);
                v = bd.gemm(Zb, Qt[BR], hbL, hbR, vrB, vrB, 1, 1, vrB, P1);
                if (!path_norms) den_cross[5] = pg.norm_slot;
                if (den_cross[5] < 0)
                    den_cross[5] = pg.tensors[bd.gemm(Qt[BL], Qt[BR], hbL, hbR, vrB, vrB, 1, 1, vrB, Mtop)].slot;
                pg.zz_den[bi] = den_cross[5];
            } else {
                throw std::logic_error("pair between unknown corners");
            }
            return v;
        };
        pg.zz_slot.assign(bonds.size(), -1);
        pg.zz_den.assign(bonds.size(), pg.norm_slot);
        // the pairs in corner order: a.q <= b.q, and a.t < b.t inside one corner
        struct Pair { SiteRef a, b; int opa, opb; };
        std::vector<Pair> pr(bonds.size());
        for (size_t bi = 0; bi < bonds.size(); ++bi) {
            if (bonds[bi].a == bonds[bi].b || bonds[bi].a < 0 || bonds[bi].b < 0 || bonds[bi].a >= nsite ||
                bonds[bi].b >= nsite)
                throw std::invalid_argument("a pair needs two distinct sites of the lattice");
            Pair& p = pr[bi];
            p.a = where[bonds[bi].a]; p.b = where[bonds[bi].b];
            p.opa = bonds[bi].op_a; p.opb = bonds[bi].op_b;
            if (p.a.q > p.b.q || (p.a.q == p.b.q && p.a.t > p.b.t)) {
                std::swap(p.a, p.b);
                std::swap(p.opa, p.opb);
            }
        }
        auto max_out = [&](int q, int t0, int t1) {
            int64_t m = 0;
            for (int u = t0; u <= t1; ++u) m = std::max(m, step_of(q, u).n_out);
            return m;
        };
        // Chains run in stages: a chain whose temporaries would push the stage
        // above kStageElems starts after every earlier chain has finished, so
        // the arena reuses their memory (only the amount of concurrent work
        // changes, not any value).
        constexpr int64_t kStageElems = int64_t(1) << 27;
        if (!recompute) {
            // sites
            for (int s = 0; s < (with_sites ? nsite : 0); ++s)
                emit_site(s, F[where[s].q][where[s].t - 1], G[where[s].q][where[s].t]);
            int64_t stage_used = 0;
            int stage_floor = 0, stage_end = 0;
            auto begin_chain = [&](int64_t temp) {
                if (stage_used > 0 && stage_used + temp > kStageElems) {
                    stage_floor = stage_end;
                    stage_used = 0;
                }
                stage_used += temp;
                bd.set_floor(stage_floor);
            };
            auto end_chain = [&](int last_tensor) {
                stage_end = std::max(stage_end, pg.tensors[last_tensor].level);
                bd.set_floor(0);
            };
            for (size_t bi = 0; bi < bonds.size(); ++bi) {
                const Pair& p = pr[bi];
                int v = -1;
                if (p.a.q == p.b.q) {
                    const int q = p.a.q;
                    begin_chain(2 * max_out(q, p.a.t, p.b.t));
                    v = chain(q, F[q][p.a.t - 1], p.a.t, p.b.t, G[q][p.b.t], p.opa, p.opb);
                    end_chain(v);
                    pg.zz_den[bi] = norm_at(q, p.b.t, G[q][p.b.t], {});
                } else {
                    const int Ta = (int)pl.corner[p.a.q].steps.size(), Tb = (int)pl.corner[p.b.q].steps.size();
                    begin_chain(2 * max_out(p.a.q, p.a.t, Ta) + 2 * max_out(p.b.q, p.b.t, Tb));
                    v = emit_cross(bi, p.a.q, p.a.t, p.opa, p.b.q, p.b.t, p.opb, F[p.a.q][p.a.t - 1],
                                   F[p.b.q][p.b.t - 1]);
                    end_chain(v);
                }
                pg.zz_slot[bi] = pg.tensors[v].slot;
            }
        } else {
            // Recompute form.  The forward chains keep only the states that
            // start a frame row (and the finished corners); every other state
            // is absorbed again from the checkpoint before it where an
            // observable needs it.  Corner by corner, the environment sweep
            // runs from the ring back to the corner's first step, holding one
            // G[q][t] at a time, and every observable whose environment is
            // G[q][t] is formed before the sweep moves on.
            auto is_ckpt = [&](int q, int t) {
                const int T = (int)pl.corner[q].steps.size();
                return t == 0 || t == T || step_of(q, t + 1).c == 0;
            };
            auto ckpt_before = [&](int q, int t) {
                while (!is_ckpt(q, t)) --t;
                return t;
            };
            // F[q][t]: the checkpoint, then single steps (the forward chain's own ops)
            auto F_at = [&](int q, int t) {
                const int u = ckpt_before(q, t);
                int x = F[q][u];
                for (int v = u + 1; v <= t; ++v) x = bd.absorb(x, E_at(q, v, PH_I), step_of(q, v), false);
                return x;
            };
            // a stage holds about two of the largest chain states: small
            // observables still share a stage, large ones run one at a time
            const int64_t stage_elems = std::min(kStageElems, 2 * pl.peak);
            int64_t used = 0;
            int stage_floor = 0;
            auto stage = [&](int64_t temp) {
                if (used > 0 && used + temp > stage_elems) {
                    stage_floor = bd.max_level();
                    used = 0;
                }
                used += temp;
                bd.set_gfloor(stage_floor);
            };
            // temporaries of a chain from the checkpoint before step t0 through step t1
            auto chain_temp = [&](int q, int t0, int t1) {
                const int u = ckpt_before(q, t0 - 1);
                return 2 * max_out(q, std::max(u, 1), std::max(t1, 1));
            };
            std::vector<std::vector<size_t>> inner(4 * (nsite + 1));
            std::vector<size_t> cross;
            for (size_t bi = 0; bi < bonds.size(); ++bi) {
                if (pr[bi].a.q == pr[bi].b.q) inner[pr[bi].b.q * (nsite + 1) + pr[bi].b.t].push_back(bi);
                else cross.push_back(bi);
            }
            for (int q = 0; q < 4; ++q) {
                const int T = (int)pl.corner[q].steps.size();
                if (!T) continue;
                stage(stage_elems);
                int Gt = env_of(q);
                for (int t = T; t >= 1; --t) {
                    const int64_t nt = step_of(q, t).n_out;
                    if (with_sites) {
                        stage(chain_temp(q, t, t) + nt);
                        emit_site(site_of(q, t), F_at(q, t - 1), Gt);
                    }
                    for (size_t bi : inner[q * (nsite + 1) + t]) {
                        const Pair& p = pr[bi];
                        stage(chain_temp(q, p.a.t, t) + nt);
                        const int v = chain(q, F_at(q, p.a.t - 1), p.a.t, t, Gt, p.opa, p.opb);
                        pg.zz_slot[bi] = pg.tensors[v].slot;
                        pg.zz_den[bi] = norm_at(q, t, Gt, [&] { return F_at(q, t - 1); });
                    }
                    if (t >= 2) {
                        stage(step_of(q, t).n_in + nt);
                        Gt = bd.absorb(Gt, E_at(q, t, PH_I), step_of(q, t), true);
                    }
                }
            }
            // pairs across the cuts, one class after another (the cached
            // products of a class die before the next class starts)
            auto cls = [&](size_t bi) { return pr[bi].a.q * 4 + pr[bi].b.q; };
            std::stable_sort(cross.begin(), cross.end(), [&](size_t x, size_t y) { return cls(x) < cls(y); });
            for (size_t bi : cross) {
                const Pair& p = pr[bi];
                const int Ta = (int)pl.corner[p.a.q].steps.size(), Tb = (int)pl.corner[p.b.q].steps.size();
                stage(chain_temp(p.a.q, p.a.t, Ta) + chain_temp(p.b.q, p.b.t, Tb));
                const int v = emit_cross(bi, p.a.q, p.a.t, p.opa, p.b.q, p.b.t, p.opb, F_at(p.a.q, p.a.t - 1),
                                         F_at(p.b.q, p.b.t - 1));
                pg.zz_slot[bi] = pg.tensors[v].slot;
            }
            bd.set_gfloor(0);
        }
    }
    int nl = 0;
    for (const auto& op : pg.ops) nl = std::max(nl, op.level);
    pg.n_levels = nl + 1;
    pg.arena_bytes = pack_arena(pg);
    return pgp;
}

std::string program_verify(const Program& pg) {
    const auto& T = pg.tensors;
    auto bad_id = [&](int id) { return id < 0 || id >= (int)T.size(); };
    // waves: every op runs after the ops that produce its inputs, at its outputs' wave
    for (size_t k = 0; k < pg.ops.size(); ++k) {
        const Op& op = pg.ops[k];
        for (int in : {op.in, op.E, op.E2, op.E3, op.adj, op.A, op.B, op.C}) {
            if (in < 0) continue;
            if (bad_id(in)) return "op " + std::to_string(k) + " reads an unknown tensor";
            const Tensor& t = T[in];
            if (t.level >= op.level && !t.is_site)
                return "op " + std::to_string(k) + " reads a tensor produced at its own or a later wave";
            if (t.last_use < op.level) return "op " + std::to_string(k) + " reads a tensor after its last use";
        }
        for (int o : {op.out, op.out2, op.out3}) {
            if (o < 0) continue;
            if (bad_id(o)) return "op " + std::to_string(k) + " writes an unknown tensor";
            if (T[o].level != op.level) return "op " + std::to_string(k) + " writes outside its wave";
        }
    }
    // arena: tensors alive in a common wave never share bytes, all lie inside it
    struct Iv { int64_t lo, hi; int l0, l1; };
    std::vector<Iv> iv;
    for (const Tensor& t : T) {
        if (t.n == 0 || t.is_site) continue;
        const int64_t len = t.n * pg.esize;
        if (t.offset < 0 || t.offset + len > pg.arena_bytes) return "tensor outside the arena";
        iv.push_back({t.offset, t.offset + len, t.level, std::max(t.level, t.last_use)});
    }
    std::sort(iv.begin(), iv.end(), [](const Iv& a, const Iv& b) { return a.lo < b.lo; });
    for (size_t a = 0; a < iv.size(); ++a)
        for (size_t b = a + 1; b < iv.size() && iv[b].lo < iv[a].hi; ++b)
            if (iv[a].l0 <= iv[b].l1 && iv[b].l0 <= iv[a].l1) return "two live tensors share arena bytes";
    return "";
}

}  // namespace tn
