"""The paper's contraction-order heuristic, written plainly -- TEST INFRASTRUCTURE ONLY.

Sec. 4: the network is contracted as a chain of pairwise contractions; the
size of a pairwise result follows d(B) = d(A1) d(A2) / d(x) (x = shared legs)
and the largest intermediate is the bottleneck contraction.  The heuristic
picks the contraction order with the smallest bottleneck and splits the
lattice into parts around the ring that closes the contraction.  The
candidates are the row scheme (Fig. 2a), the quadrant scheme (Fig. 2b) and
the cuts that lie between the two.

Reading used here (the paper gives no formula for the candidates):
  * orientation o in {0, 1}: o = 1 works on the transposed lattice
    (L' = W, W' = L), o = 0 on the lattice itself;
  * a cut (i, j), 0 <= i <= L', 0 <= j <= W', splits the lattice into the four
    corners TL = rows [0,i) x cols [0,j), TR = rows [0,i) x cols [j,W'),
    BL = rows [i,L') x cols [0,j), BR = rows [i,L') x cols [j,W'); (L', W')
    is the row scheme, the middle cut is the quadrant scheme, every other cut
    lies in between;
  * each corner is grown row by row from its outer lattice corner, one site at
    a time, in the corner's mirrored frame (TR mirrors columns, BL mirrors
    rows, BR both), keeping its boundary legs in the order
    [dn_0 .. dn_{c-1}, h, u_c .. u_{b-1}, rt_{k-1} .. rt_0];
  * the ring of four corners is closed by M_top = TL TR^T, M_bot = BL BR^T and
    <M_top, M_bot>;
  * bottleneck = the largest input or output (in entries, double layer,
    d = D^2 per bond) of any of these pairwise contractions;
  * ties: fewest multiply-adds, then the cut nearest the middle
    (|2i - L'| + |2j - W'|), then o, then i, then j (all smallest first);
    for an energy evaluation, whose environment method keeps every chain
    state, the summed size of all chain-step outputs is compared right after
    the bottleneck;
  * integer products and sums saturate at 2^62 (such plans never fit memory).

Forced schedules: ROW = (o=0, i=L, j=W); COL = (o=1, i=W, j=L);
QUADRANT = (o=0, i=ceil(L/2), j=ceil(W/2)).
"""
from __future__ import annotations

CAP = 1 << 62
AUTO, ROW, COL, QUADRANT = 0, 1, 2, 3


def _mul(a: int, b: int) -> int:
    return min(a * b, CAP)


def _add(a: int, b: int) -> int:
    return min(a + b, CAP)


def _pow(d: int, n: int) -> int:
    v = 1
    for _ in range(n):
        v = _mul(v, d)
    return v


def _corner_steps(q: int, o: int, i: int, j: int, Lp: int, Wp: int, d: int):
    """Chain of corner q (0 TL, 1 TR, 2 BL, 3 BR) as a list of step dicts."""
    a = i if q in (0, 1) else Lp - i
    b = j if q in (0, 2) else Wp - j
    if a == 0 or b == 0:
        return []
    if q in (0, 1):
        bottom = d if i < Lp else 1
    else:
        bottom = d if i > 0 else 1
    if q in (0, 2):
        right = d if j < Wp else 1
    else:
        right = d if j > 0 else 1

    def fu(k, c):
        return 1 if k == 0 else d

    def fl(k, c):
        return 1 if c == 0 else d

    def fdn(k, c):
        return d if k < a - 1 else bottom

    def frt(k, c):
        return d if c < b - 1 else right

    steps = []
    for k in range(a):
        for c in range(b):
            P = 1
            for cc in range(c):
                P = _mul(P, fdn(k, cc))
            S = 1
            for cc in range(c + 1, b):
                S = _mul(S, fu(k, cc))
            for kk in range(k):
                S = _mul(S, frt(kk, b - 1))
            K = fl(k, c) * fu(k, c)
            N = fdn(k, c) * frt(k, c)
            # oriented-lattice coordinates of this frame site
            rr = k if q in (0, 1) else Lp - 1 - k
            cc_ = c if q in (0, 2) else Wp - 1 - c
            r, col = (rr, cc_) if o == 0 else (cc_, rr)
            steps.append(dict(corner=q, k=k, c=c, r=r, col=col, P=P, K=K, N=N, S=S,
                              n_in=_mul(_mul(P, K), S), n_out=_mul(_mul(P, N), S),
                              mac=_mul(_mul(_mul(P, S), K), N)))
    return steps


def evaluate(L: int, W: int, D: int, o: int, i: int, j: int) -> dict:
    d = D * D
    Lp, Wp = (L, W) if o == 0 else (W, L)
    steps = []
    for q in range(4):
        steps += _corner_steps(q, o, i, j, Lp, Wp, d)
    hcut = d if 0 < i < Lp else 1
    vcut = d if 0 < j < Wp else 1
    m_size = _pow(hcut, Wp)
    peak = m_size
    mac = 0
    cached = 0
    for s in steps:
        peak = max(peak, s["n_in"], s["n_out"])
        mac = _add(mac, s["mac"])
        cached = _add(cached, s["n_out"])
    mac = _add(mac, _mul(m_size, _pow(vcut, i)))        # M_top = TL TR^T
    mac = _add(mac, _mul(m_size, _pow(vcut, Lp - i)))   # M_bot = BL BR^T
    mac = _add(mac, m_size)                             # <M_top, M_bot>
    return dict(o=o, i=i, j=j, peak=peak, mac=mac, steps=steps, cached=cached,
                centre=abs(2 * i - Lp) + abs(2 * j - Wp))


def plan(L: int, W: int, D: int, schedule: int = AUTO, energy: bool = False) -> dict:
    if schedule == ROW:
        return evaluate(L, W, D, 0, L, W)
    if schedule == COL:
        return evaluate(L, W, D, 1, W, L)
    if schedule == QUADRANT:
        return evaluate(L, W, D, 0, (L + 1) // 2, (W + 1) // 2)
    best, best_key = None, None
    for o in (0, 1):
        Lp, Wp = (L, W) if o == 0 else (W, L)
        for i in range(Lp + 1):
            for j in range(Wp + 1):
                ev = evaluate(L, W, D, o, i, j)
                key = (ev["peak"], ev["cached"] if energy else 0, ev["mac"], ev["centre"], o, i, j)
                if best_key is None or key < best_key:
                    best, best_key = ev, key
    return best
