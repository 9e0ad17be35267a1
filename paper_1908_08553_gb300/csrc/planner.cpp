// Partition and contraction-order choice of Sec. 4: among the candidate
// partitions, take the one whose largest pairwise contraction (the bottleneck)
// is smallest and split the lattice into corners around the closing ring,
// with the size rule d(B) = d(A1) d(A2) / d(x) of the same section applied to
// every site absorption and ring product.
//
// Candidates: orientation o (o = 1: transposed lattice) and a cut (i, j) of
// the oriented Lp x Wp lattice into corners TL, TR, BL, BR (rows [0,i) /
// [i,Lp), columns [0,j) / [j,Wp)).  (Lp, Wp) is the row scheme of Fig. 2a, the
// middle cut the quadrant scheme of Fig. 2b, the rest the cuts in between.
// Each corner grows row by row from its outer lattice corner in a mirrored
// frame (TR mirrors columns, BL rows, BR both), its boundary legs ordered
// [dn_0..dn_{c-1}, h, u_c..u_{b-1}, rt_{k-1}..rt_0]; the ring closes as
// M_top = TL TR^T, M_bot = BL BR^T, <M_top, M_bot>.
// Bottleneck = largest input or output (entries) of those contractions; ties
// go to fewer multiply-adds, then the cut nearest the middle, then smaller o,
// i, j.  For energies (which keep every chain state for the environment
// method) the second key is the summed size of the chain outputs.  Integer
// arithmetic saturates at 2^62.
#include <algorithm>
#include <climits>

#include "tn_internal.h"

namespace tn {

namespace {

int64_t ipow_sat(int64_t d, int n) {
    int64_t v = 1;
    for (int k = 0; k < n; ++k) v = sat_mul(v, d);
    return v;
}

// Leg roles: 0 u, 1 l, 2 dn, 3 rt.
void frame_map(int o, int q, int* map) {
    // oriented leg -> original leg
    int om[4] = {0, 1, 2, 3};
    if (o == 1) { om[0] = 1; om[1] = 0; om[2] = 3; om[3] = 2; }
    // frame leg -> oriented leg
    int fm[4] = {0, 1, 2, 3};
    if (q == TR || q == BR) std::swap(fm[1], fm[3]);
    if (q == BL || q == BR) std::swap(fm[0], fm[2]);
    for (int k = 0; k < 4; ++k) map[k] = om[fm[k]];
}

}  // namespace

void orient(const Plan& p, int r, int c, int* rr, int* cc) {
    if (p.o == 0) { *rr = r; *cc = c; } else { *rr = c; *cc = r; }
}

Plan plan_evaluate(int L, int W, int D, int o, int i, int j) {
    Plan p;
    p.L = L; p.W = W; p.D = D; p.d = D * D;
    p.o = o; p.i = i; p.j = j;
    p.Lp = o == 0 ? L : W;
    p.Wp = o == 0 ? W : L;
    const int d = p.d, Lp = p.Lp, Wp = p.Wp;
    const int hcut = (i > 0 && i < Lp) ? d : 1;
    const int vcut = (j > 0 && j < Wp) ? d : 1;
    p.hb_L = ipow_sat(hcut, j);
    p.hb_R = ipow_sat(hcut, Wp - j);
    p.vr_T = ipow_sat(vcut, i);
    p.vr_B = ipow_sat(vcut, Lp - i);
    int64_t peak = 0, mac = 0;
    for (int q = 0; q < 4; ++q) {
        CornerPlan& cp = p.corner[q];
        const bool top = (q == TL || q == TR), left = (q == TL || q == BL);
        cp.a = top ? i : Lp - i;
        cp.b = left ? j : Wp - j;
        cp.bottom = top ? (i < Lp ? d : 1) : (i > 0 ? d : 1);
        cp.right = left ? (j < Wp ? d : 1) : (j > 0 ? d : 1);
        frame_map(o, q, cp.map);
        cp.size_b = ipow_sat(cp.bottom, cp.b);
        cp.size_r = ipow_sat(cp.right, cp.a);
        if (cp.a == 0 || cp.b == 0) { cp.size_b = cp.size_r = 1; continue; }
        const int a = cp.a, b = cp.b;
        // double-layer leg dims in the frame
        auto du = [&](int k) { return k == 0 ? 1 : d; };
        auto dl = [&](int c) { return c == 0 ? 1 : d; };
        auto ddn = [&](int k) { return k < a - 1 ? d : cp.bottom; };
        auto drt = [&](int c) { return c < b - 1 ? d : cp.right; };
        // S grows by the rt leg each finished row contributes
        int64_t rt_done = 1;
        for (int k = 0; k < a; ++k) {
            for (int c = 0; c < b; ++c) {
                Step s;
                s.corner = q; s.k = k; s.c = c;
                int orr = top ? k : Lp - 1 - k;
                int occ = left ? c : Wp - 1 - c;
                if (o == 0) { s.r = orr; s.col = occ; } else { s.r = occ; s.col = orr; }
                s.P = ipow_sat(ddn(k), c);                  // dn legs already emitted in this row
                s.S = sat_mul(ipow_sat(du(k), b - 1 - c), rt_done);
                s.K = dl(c) * du(k);
                s.N = ddn(k) * drt(c);
                s.n_in = sat_mul(sat_mul(s.P, s.K), s.S);
                s.n_out = sat_mul(sat_mul(s.P, s.N), s.S);
                s.mac = sat_mul(sat_mul(sat_mul(s.P, s.S), s.K), s.N);
                peak = std::max(peak, std::max(s.n_in, s.n_out));
                mac = sat_add(mac, s.mac);
                p.chain_elems = sat_add(p.chain_elems, s.n_out);
                cp.steps.push_back(s);
            }
            rt_done = sat_mul(rt_done, drt(b - 1));
        }
    }
    const int64_t m_size = sat_mul(p.hb_L, p.hb_R);
    peak = std::max(peak, m_size);
    mac = sat_add(mac, sat_mul(m_size, p.vr_T));
    mac = sat_add(mac, sat_mul(m_size, p.vr_B));
    mac = sat_add(mac, m_size);
    p.peak = peak;
    p.mac = mac;
    p.centre = std::abs(2 * i - Lp) + std::abs(2 * j - Wp);
    return p;
}

Plan plan_choose(int L, int W, int D, tn_schedule sched, tn_work work) {
    switch (sched) {
        case TN_SCHED_ROW: return plan_evaluate(L, W, D, 0, L, W);
        case TN_SCHED_COL: return plan_evaluate(L, W, D, 1, W, L);
        case TN_SCHED_QUADRANT: return plan_evaluate(L, W, D, 0, (L + 1) / 2, (W + 1) / 2);
        default: break;
    }
    Plan best;
    bool have = false;
    for (int o = 0; o < 2; ++o) {
        const int Lp = o == 0 ? L : W, Wp = o == 0 ? W : L;
        for (int i = 0; i <= Lp; ++i)
            for (int j = 0; j <= Wp; ++j) {
                Plan c = plan_evaluate(L, W, D, o, i, j);
                // energies cache every chain state: among cuts with the same
                // bottleneck they prefer the smallest cached total
                const int64_t kc = work != TN_WORK_NORM ? c.chain_elems : 0;
                const int64_t kb = work != TN_WORK_NORM ? best.chain_elems : 0;
                auto key = std::make_tuple(c.peak, kc, c.mac, c.centre, c.o, c.i, c.j);
                auto bkey = std::make_tuple(best.peak, kb, best.mac, best.centre, best.o, best.i, best.j);
                if (!have || key < bkey) { best = std::move(c); have = true; }
            }
    }
    return best;
}

}  // namespace tn
