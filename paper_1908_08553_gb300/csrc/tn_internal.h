// Internal declarations of libtn (host side).  Not part of the C-ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/tn.h"

namespace tn {

constexpr int64_t kCap = int64_t(1) << 62;   // saturation bound of planner integers

inline int64_t sat_mul(int64_t a, int64_t b) {
    if (a == 0 || b == 0) return 0;
    if (a > kCap / b) return kCap;
    int64_t v = a * b;
    return v > kCap ? kCap : v;
}
inline int64_t sat_add(int64_t a, int64_t b) {
    int64_t v = a + b;
    return v > kCap ? kCap : v;
}

// ------------------------------------------------------------------ plan --

// Corners of the ring (Sec. 4, quadrant scheme) in the oriented lattice.
enum Corner { TL = 0, TR = 1, BL = 2, BR = 3 };

// One site absorption: boundary [P, K, S] -> [P, N, S].
struct Step {
    int corner, k, c;        // frame row / column inside the corner
    int r, col;              // lattice site (original orientation)
    int64_t P, S;
    int K, N;
    int64_t n_in, n_out, mac;
};

struct CornerPlan {
    int a = 0, b = 0;        // frame rows / columns
    int bottom = 1, right = 1;   // double-layer dims of the frame's bottom / right cut legs
    int map[4] = {0, 1, 2, 3};   // frame leg role (u,l,dn,rt) -> original leg index
    std::vector<Step> steps;     // chain order
    int64_t size_b = 1, size_r = 1;   // final tensor as [size_b][size_r]
};

struct Plan {
    int L = 0, W = 0, D = 0, d = 0;
    int o = 0, i = 0, j = 0;     // orientation and cut
    int Lp = 0, Wp = 0;          // oriented lattice dims
    int64_t peak = 0, mac = 0;
    int64_t chain_elems = 0;     // summed outputs of all chain steps (what an energy caches)
    int centre = 0;
    CornerPlan corner[4];
    int64_t hb_L = 1, hb_R = 1, vr_T = 1, vr_B = 1;   // ring leg-group sizes
};

Plan plan_evaluate(int L, int W, int D, int o, int i, int j);
Plan plan_choose(int L, int W, int D, tn_schedule sched, tn_work work = TN_WORK_NORM);
// oriented coordinates (r', c') of lattice site (r, c)
void orient(const Plan& p, int r, int c, int* rr, int* cc);

// ---------------------------------------------------------------- program --

enum DType { DT_F64 = 0, DT_F32 = 1 };

enum OpKind {
    OP_SITEMAT = 0,   // build a double-layer site matrix E (K x N)
    OP_ABSORB,        // out = absorb(in, E)        [P,K,S] -> [P,N,S]
    OP_ABSORB_DOT,    // scalar = <absorb(in, E), adj>
    OP_GEMM,          // C = opA(A) opB(B)
    OP_GEMM_DOT,      // scalar = <opA(A) opB(B), C>
    OP_DOT,           // scalar = <A, B>
    OP_TC_SPLIT,      // FP32 operand -> tiled BF16 planes (tensor-core input)
    OP_TC_GEMM,       // C = A B^T on tensor cores from split planes
    OP_TC_GEMM_DOT,   // scalar = <A B^T, C> on tensor cores
    OP_ABSORB2,       // out = absorb(absorb(in, E), E2): two steps of one frame row
    OP_ABSORB2_DOT,   // scalar = <absorb(absorb(in, E), E2), adj>
};

// Operator insertion on the physical leg.
// PH_R = [[0, 1], [-1, 0]]: Y = i R on this basis, so a real state's <Y_i Y_j>
// is -<R_i R_j> (and any single Y averages to zero).  PH_Y = [[0, i], [-i, 0]]
// itself, for complex site tensors only (their site matrices are built from
// complex arithmetic, see k_sitemat).
enum PhysOp { PH_I = 0, PH_X = 1, PH_Z = 2, PH_R = 3, PH_Y = 4 };

// One two-site correlator <A_a B_b> of an explicit pair list (sites row-major).
struct PairSpec {
    int a, b, op_a, op_b;
};

struct Tensor {
    int64_t n = 0;           // entries (0 for a scalar result)
    int64_t offset = -1;     // bytes into the arena
    int slot = -1;           // exponent / max / scalar slot
    int level = 0;           // wave that produces it
    int last_use = -1;       // last wave that reads it
    bool is_const_one = false;
    bool is_site = false;    // raw FP64 site tensor (lattice input), offset into the input area
    int site = -1;
    bool factored = false;   // site matrix kept as its two layer factors (interior D = 3 steps)
};

struct Op {
    OpKind kind;
    int level = 0;
    // absorb
    int in = -1, E = -1, out = -1, adj = -1;
    int E2 = -1, out2 = -1;       // dual / triple absorb-dot: second site matrix and its scalar
    int E3 = -1, out3 = -1;       // triple absorb-dot: third site matrix and its scalar
    int64_t P = 0, S = 0;
    int K = 0, N = 0;
    bool transE = false;
    // gemm: C[m][n] = sum_k A(m,k) B(k,n); A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]
    int A = -1, B = -1, C = -1;
    int64_t gm = 0, gn = 0, gk = 0;
    int64_t sam = 0, sak = 0, sbk = 0, sbn = 0;
    // tensor cores: source tensors of the split operands (their slots carry the scale)
    int A_src = -1, B_src = -1;
    int nsplit = 0;               // tensor cores: 2 or 3 split planes (products and D=3 absorption)
    bool factored = false;        // sitemat: write the layer factors; absorb: ket pass then bra pass
    long long Rp = 0, Kp = 0;
    // sitemat
    int site = -1, phys = PH_I;
    int map[4] = {0, 1, 2, 3};
    int fdim[4] = {1, 1, 1, 1};  // frame dims (u, l, dn, rt), single layer
    // algorithmic accounting
    double bytes = 0, macs = 0;
};

// Choices the program builder makes per lattice shape: each is exact (the
// values computed are the same to rounding), only speed differs, so an
// autotuner times them (autotune.cpp).  The defaults are the fixed rules.
struct Knobs {
    bool fuse_pairs = true;     // FP32 D = 2: two steps of a frame row in one pass (OP_ABSORB2)
    bool site_triple = true;    // FP32 D <= 2: <X_k>, <Z_k> and the local norm in one absorb-dot
    bool factor_d3 = true;      // D = 3 interior steps: ket pass then bra pass (off: the double-layer
                                // matrix, on the tensor cores in the split-BF16 precisions)
    bool tc_products = true;    // BF16x3 / BF16x6: products of >= 2^26 multiply-adds on the tensor cores
    bool tc_small = false;      // ... and the smaller ones too (else FP32 SIMT)
    bool recompute = false;     // energies: keep only the chain states that start a frame row and
                                // recompute the others where an observable needs them, one
                                // observable after another (memory-bounded; the same ops on the
                                // same inputs, so the same bits)
    int code() const {
        return (fuse_pairs ? 1 : 0) | (site_triple ? 2 : 0) | (factor_d3 ? 4 : 0) | (tc_products ? 8 : 0) |
               (tc_small ? 16 : 0) | (recompute ? 32 : 0);
    }
    static Knobs from_code(int c) {
        Knobs k;
        k.fuse_pairs = c & 1; k.site_triple = c & 2; k.factor_d3 = c & 4; k.tc_products = c & 8;
        k.tc_small = c & 16; k.recompute = c & 32;
        return k;
    }
};
constexpr int kDefaultKnobs = 15;
constexpr int kMaxKnobs = 63;
constexpr int kRecomputeKnob = 32;

// Result addressing inside one program: which scalar slots hold what.
struct Program {
    Plan plan;
    tn_work work = TN_WORK_ENERGY;
    Knobs knobs;
    DType dt = DT_F32;
    int nsplit = 0;               // 2 or 3: dense products on tensor cores (BF16 split)
    int esize = 4;
    std::vector<Tensor> tensors;
    std::vector<Op> ops;
    int n_levels = 0;
    int norm_slot = -1;
    std::vector<int> sx_slot;     // per site (row-major, original lattice)
    std::vector<int> zz_slot;     // per bond (output order)
    std::vector<int> sz_slot;     // per site: <Z_k> numerator (denominator sx_den)
    std::vector<int> sy_slot;     // complex site tensors: per site <Y_k> numerator (denominator sx_den)
    bool cplx = false;            // complex site tensors: per site the real parts, then the imaginary parts
    // denominator of each ratio: <F[q][t], G[q][t]> at the step where the
    // observable meets its environment (the norm along the same rounding path),
    // or norm_slot for bonds across a cut
    std::vector<int> sx_den, zz_den;
    int n_slots = 0;
    int64_t arena_bytes = 0;      // tensors + site matrices (typed)
    int64_t input_bytes = 0;      // raw FP64 site tensors
    std::vector<int64_t> site_offset;   // FP64 entries, per site
    std::vector<int> site_dims;          // 4 per site
};

// Internal work kinds beyond tn_work: the nearest-neighbour correlators
// <A_i B_j> alone, A = PhysOp a and B = PhysOp b (X, Z, R or Y).
inline tn_work work_bonds(int a, int b) { return (tn_work)(16 + 8 * a + b); }
inline bool work_is_bonds(tn_work w) { return (int)w >= 16; }
inline int work_bond_a(tn_work w) { return ((int)w - 16) / 8; }
inline int work_bond_b(tn_work w) { return ((int)w - 16) % 8; }
inline bool work_valid(tn_work w) {
    if (w == TN_WORK_NORM || w == TN_WORK_ENERGY) return true;
    if (!work_is_bonds(w) || (int)w >= 16 + 8 * 8) return false;
    const int a = work_bond_a(w), b = work_bond_b(w);
    auto ok = [](int o) { return o == PH_X || o == PH_Z || o == PH_R || o == PH_Y; };
    return ok(a) && ok(b);
}

// cplx: complex site tensors (the input layout and the site matrices change,
// nothing downstream of them does)
std::shared_ptr<const Program> program_build(int L, int W, int D, tn_schedule sched,
                                             tn_precision prec, tn_work work, Knobs knobs = Knobs(),
                                             bool cplx = false);
// the same for a given plan (any orientation and cut)
// pairs (work TN_WORK_ENERGY): the correlators of that list instead of the
// energy's observables (result order = list order)
std::shared_ptr<const Program> program_build_plan(const Plan& plan, tn_precision prec, tn_work work,
                                                  Knobs knobs = Knobs(),
                                                  const std::vector<PairSpec>* pairs = nullptr,
                                                  bool cplx = false);
// Knobs the tuning table holds for this shape (the defaults if it holds none).
Knobs tuned_knobs(int L, int W, int D, tn_precision prec, tn_work work);
// Consistency of a built program ("" if sound): every op runs after the
// producers of its inputs and within their lifetimes, and no two tensors alive
// in a common wave share arena bytes.
std::string program_verify(const Program& pg);

}  // namespace tn
