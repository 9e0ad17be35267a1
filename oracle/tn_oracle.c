/*
 * tn_oracle.c -- plain, slow FP64 CPU oracle for the exact contraction of an
 * open-boundary PEPS of the transverse-field Ising model.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this code.  It shares no code, header, table or helper
 * with the CUDA library: it takes the same seeded site tensors as input and
 * nothing else.
 *
 * What it computes (Sec. 3, Eqs. norm, Etot, mx, cij; Sec. 5 on which networks
 * are contracted):
 *   norm      <Psi|Psi> = sum_sigma A(sigma)^2       (amplitudes are real, Sec. 3)
 *   <sx_k>    <Psi|X_k|Psi> / <Psi|Psi>             (Eq. mx with S^x = X)
 *   <zz_ij>   <Psi|Z_i Z_j|Psi> / <Psi|Psi>         (first term of Eq. cij)
 *   E         -J sum_<ij> <zz_ij> - h sum_k <sx_k>  (Eqs. Hamiltonian and Etot)
 * with Pauli operators (spins +-1, Sec. 3), Z = diag(-1, +1) on p = 0, 1 because
 * p = 1 is sigma = +1 (x = (sigma + 1)/2, Eq. Psi).
 *
 * How: the "row" order of Sec. 4 -- the network is swept row by row from one
 * edge to the other, one site tensor at a time, keeping the full boundary
 * tensor (no truncation; the method is exact, Abstract and Sec. 1).  Top
 * boundaries T_r (rows 0..r-1 absorbed) and bottom boundaries B_r (rows
 * L-1..r absorbed) are cached, so
 *   norm          = <T_r, B_r>                        for every r,
 *   site (r,c)    = <T_r + row r with X at c, B_{r+1}>,
 *   bond (r,c)-(r,c+1) = <T_r + row r with Z at c, c+1, B_{r+1}>,
 *   bond (r,c)-(r+1,c) = <T_r + rows r, r+1 with Z at column c, B_{r+2}>.
 * Every boundary is kept as a mantissa array times 2^e; after each absorbed
 * site the array is rescaled by an exact power of two so the norm of a large
 * lattice cannot overflow.
 *
 * Site tensors A[p][u][l][dn][rt] (C order), bond legs D or 1 on the lattice
 * edge, stored site after site in row-major site order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- grids -- */

/* A planar L x W grid of rank-4 tensors T[u][l][dn][rt]. */
typedef struct {
    int L, W;
    int *dim;      /* 4 per site: u, l, dn, rt */
    double **t;    /* per-site tensor */
} grid_t;

static grid_t grid_alloc(int L, int W) {
    grid_t g;
    g.L = L; g.W = W;
    g.dim = (int *)calloc((size_t)4 * L * W, sizeof(int));
    g.t = (double **)calloc((size_t)L * W, sizeof(double *));
    return g;
}

static void grid_free(grid_t *g) {
    for (int k = 0; k < g->L * g->W; ++k) free(g->t[k]);
    free(g->t); free(g->dim);
}

static size_t tsize(const int *d) { return (size_t)d[0] * d[1] * d[2] * d[3]; }

/* Mirror the grid top <-> bottom: new row r is old row L-1-r, u and dn swap. */
static grid_t grid_flip_rows(const grid_t *g) {
    grid_t f = grid_alloc(g->L, g->W);
    for (int r = 0; r < g->L; ++r)
        for (int c = 0; c < g->W; ++c) {
            int so = (g->L - 1 - r) * g->W + c, sn = r * g->W + c;
            const int *d = g->dim + 4 * so;
            int *e = f.dim + 4 * sn;
            e[0] = d[2]; e[1] = d[1]; e[2] = d[0]; e[3] = d[3];
            f.t[sn] = (double *)malloc(tsize(d) * sizeof(double));
            for (int u = 0; u < d[0]; ++u)
                for (int l = 0; l < d[1]; ++l)
                    for (int n = 0; n < d[2]; ++n)
                        for (int q = 0; q < d[3]; ++q)
                            f.t[sn][((n * d[1] + l) * d[0] + u) * d[3] + q] =
                                g->t[so][((u * d[1] + l) * d[2] + n) * d[3] + q];
        }
    return f;
}

/* ------------------------------------------------------------ boundary -- */

typedef struct {
    double *v;
    size_t n;
    int64_t e;     /* value = v * 2^e */
} bnd_t;

static void rescale(bnd_t *b) {
    double mx = 0.0;
    for (size_t i = 0; i < b->n; ++i) {
        double a = fabs(b->v[i]);
        if (a > mx) mx = a;
    }
    if (mx == 0.0 || !isfinite(mx)) return;
    int ex;
    frexp(mx, &ex);
    for (size_t i = 0; i < b->n; ++i) b->v[i] = ldexp(b->v[i], -ex);
    b->e += ex;
}

/*
 * Absorb one site tensor T[u][h][dn][rt] into a boundary whose legs are
 * [P-legs, h, u, S-legs]: out[p][dn][rt][s] = sum_{h,u} in[p][h][u][s] T[u][h][dn][rt].
 * This is the pairwise contraction of Sec. 4 (shared legs x = {h, u},
 * d(out) = d(in) d(T) / d(x)^2 ... with the two shared legs summed).
 */
static void absorb(const double *in, double *out, size_t P, int Dh, int Du,
                   int Ddn, int Drt, size_t S, const double *T) {
    long long outer = (long long)(P * S);
#pragma omp parallel for schedule(static) if (outer > 2048)
    for (long long ps = 0; ps < outer; ++ps) {
        size_t p = (size_t)ps / S, s = (size_t)ps % S;
        for (int n = 0; n < Ddn; ++n)
            for (int q = 0; q < Drt; ++q) {
                double acc = 0.0;
                for (int h = 0; h < Dh; ++h)
                    for (int u = 0; u < Du; ++u)
                        acc += in[((p * Dh + h) * Du + u) * S + s] *
                               T[((size_t)(u * Dh + h) * Ddn + n) * Drt + q];
                out[((p * Ddn + n) * Drt + q) * S + s] = acc;
            }
    }
}

/*
 * Absorb row r of grid g into boundary b (legs: the u legs of row r, in column
 * order), site by site from column 0 to W-1.  `over` optionally replaces the
 * tensor of some columns of the row (operator insertions); NULL entries mean
 * the grid's own tensor.  On return b holds the dn legs of row r.
 */
static void absorb_row_part(const grid_t *g, int r, double *const *over, bnd_t *b, int ncols) {
    int W = g->W;
    for (int c = 0; c < ncols; ++c) {
        const int *d = g->dim + 4 * (r * W + c);
        const double *T = (over && over[c]) ? over[c] : g->t[r * W + c];
        size_t P = 1, S = 1;
        for (int k = 0; k < c; ++k) P *= (size_t)g->dim[4 * (r * W + k) + 2];
        for (int k = c + 1; k < W; ++k) S *= (size_t)g->dim[4 * (r * W + k) + 0];
        int Dh = d[1], Du = d[0], Ddn = d[2], Drt = d[3];
        size_t nout = P * Ddn * Drt * S;
        double *o = (double *)malloc(nout * sizeof(double));
        absorb(b->v, o, P, Dh, Du, Ddn, Drt, S, T);
        free(b->v);
        b->v = o; b->n = nout;
        rescale(b);
    }
}

static void absorb_row(const grid_t *g, int r, double *const *over, bnd_t *b) {
    absorb_row_part(g, r, over, b, g->W);
}

static bnd_t bnd_one(void) {
    bnd_t b;
    b.v = (double *)malloc(sizeof(double));
    b.v[0] = 1.0; b.n = 1; b.e = 0;
    return b;
}

static bnd_t bnd_copy(const bnd_t *a) {
    bnd_t b;
    b.n = a->n; b.e = a->e;
    b.v = (double *)malloc(a->n * sizeof(double));
    memcpy(b.v, a->v, a->n * sizeof(double));
    return b;
}

/* <a, b> as mantissa * 2^exp. */
static void bnd_dot(const bnd_t *a, const bnd_t *b, double *m, int64_t *e) {
    double acc = 0.0;
    for (size_t i = 0; i < a->n; ++i) acc += a->v[i] * b->v[i];
    *m = acc;
    *e = a->e + b->e;
}

/* T_r for r = 0..L (rows 0..r-1 absorbed); tops[r] allocated. */
static void top_boundaries(const grid_t *g, bnd_t *tops) {
    tops[0] = bnd_one();
    for (int r = 0; r < g->L; ++r) {
        tops[r + 1] = bnd_copy(&tops[r]);
        absorb_row(g, r, NULL, &tops[r + 1]);
    }
}

/* B_r for r = 0..L (rows L-1..r absorbed), legs = u legs of row r. */
static void bottom_boundaries(const grid_t *g, bnd_t *bots) {
    grid_t f = grid_flip_rows(g);
    bnd_t *ft = (bnd_t *)malloc(sizeof(bnd_t) * (g->L + 1));
    top_boundaries(&f, ft);
    /* flipped T_k has flipped rows 0..k-1 = original rows L-1..L-k absorbed */
    for (int r = 0; r <= g->L; ++r) bots[r] = ft[g->L - r];
    free(ft);
    grid_free(&f);
}

/* ------------------------------------------------------ double layer ---- */

static const double OP_I[4] = {1, 0, 0, 1};
static const double OP_X[4] = {0, 1, 1, 0};
static const double OP_Z[4] = {-1, 0, 0, 1};
/* Y = i R on the basis (p = 0 <-> -1, p = 1 <-> +1): R is real and
 * antisymmetric, so for real amplitudes <Y_i> = 0, <A_i Y_j> = 0 for A = X, Z,
 * and <Y_i Y_j> = -<R_i R_j> (the sign convention of R cancels in R R). */
static const double OP_R[4] = {0, 1, -1, 0};

/*
 * Double-layer (bra x ket) site tensor with operator O on the physical leg:
 * E[(ua ub)][(la lb)][(da db)][(ra rb)] = sum_{p,q} A[p][ua][la][da][ra] O[p][q] A[q][ub][lb][db][rb].
 * The "a" copy is the major digit of each combined leg.  Amplitudes are real,
 * so no conjugation (Sec. 3).
 */
static double *double_layer(const double *A, const int *d, const double *O) {
    int Du = d[0], Dl = d[1], Dd = d[2], Dr = d[3];
    size_t n1 = (size_t)Du * Dl * Dd * Dr;
    double *E = (double *)calloc(n1 * n1, sizeof(double));
    for (int ua = 0; ua < Du; ++ua) for (int ub = 0; ub < Du; ++ub)
    for (int la = 0; la < Dl; ++la) for (int lb = 0; lb < Dl; ++lb)
    for (int da = 0; da < Dd; ++da) for (int db = 0; db < Dd; ++db)
    for (int ra = 0; ra < Dr; ++ra) for (int rb = 0; rb < Dr; ++rb) {
        double acc = 0.0;
        for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) {
                double o = O[p * 2 + q];
                if (o == 0.0) continue;
                acc += A[(((size_t)(p * Du + ua) * Dl + la) * Dd + da) * Dr + ra] * o *
                       A[(((size_t)(q * Du + ub) * Dl + lb) * Dd + db) * Dr + rb];
            }
        size_t iu = (size_t)ua * Du + ub, il = (size_t)la * Dl + lb;
        size_t id = (size_t)da * Dd + db, ir = (size_t)ra * Dr + rb;
        E[((iu * Dl * Dl + il) * Dd * Dd + id) * Dr * Dr + ir] = acc;
    }
    return E;
}

static void site_dims(int L, int W, int D, int r, int c, int *d) {
    d[0] = r == 0 ? 1 : D;
    d[1] = c == 0 ? 1 : D;
    d[2] = r == L - 1 ? 1 : D;
    d[3] = c == W - 1 ? 1 : D;
}

/* Offsets of each site tensor in the flat input. */
static size_t *site_offsets(int L, int W, int D) {
    size_t *off = (size_t *)malloc(sizeof(size_t) * ((size_t)L * W + 1));
    off[0] = 0;
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < W; ++c) {
            int d[4];
            site_dims(L, W, D, r, c, d);
            off[r * W + c + 1] = off[r * W + c] + 2 * tsize(d);
        }
    return off;
}

/* The norm network: double-layer tensors with the identity on every site. */
static grid_t norm_grid(int L, int W, int D, const double *A) {
    grid_t g = grid_alloc(L, W);
    size_t *off = site_offsets(L, W, D);
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < W; ++c) {
            int d[4];
            site_dims(L, W, D, r, c, d);
            int *e = g.dim + 4 * (r * W + c);
            for (int k = 0; k < 4; ++k) e[k] = d[k] * d[k];
            g.t[r * W + c] = double_layer(A + off[r * W + c], d, OP_I);
        }
    free(off);
    return g;
}

/* ------------------------------------------------------------ exports --- */

/* Norm of a generic grid of rank-4 tensors (single or double layer). */
int or_grid_contract(int L, int W, const int *dims, const double *flat,
                     double *m, int64_t *e) {
    grid_t g = grid_alloc(L, W);
    size_t off = 0;
    for (int k = 0; k < L * W; ++k) {
        for (int q = 0; q < 4; ++q) g.dim[4 * k + q] = dims[4 * k + q];
        size_t n = tsize(dims + 4 * k);
        g.t[k] = (double *)malloc(n * sizeof(double));
        memcpy(g.t[k], flat + off, n * sizeof(double));
        off += n;
    }
    bnd_t b = bnd_one();
    for (int r = 0; r < L; ++r) absorb_row(&g, r, NULL, &b);
    *m = b.v[0];
    *e = b.e;
    free(b.v);
    grid_free(&g);
    return 0;
}

/* <T_r, B_r> for every r = 0..L: the same norm cut at every row. */
int or_peps_norm_all_cuts(int L, int W, int D, const double *A, double *m, int64_t *e) {
    grid_t g = norm_grid(L, W, D, A);
    bnd_t *tops = (bnd_t *)malloc(sizeof(bnd_t) * (L + 1));
    bnd_t *bots = (bnd_t *)malloc(sizeof(bnd_t) * (L + 1));
    top_boundaries(&g, tops);
    bottom_boundaries(&g, bots);
    for (int r = 0; r <= L; ++r) bnd_dot(&tops[r], &bots[r], &m[r], &e[r]);
    for (int r = 0; r <= L; ++r) { free(tops[r].v); free(bots[r].v); }
    free(tops); free(bots);
    grid_free(&g);
    return 0;
}

/* The first nrows rows of the norm network, then the first ncols sites of row
 * nrows, absorbed into the top boundary: a bounded timing sample of the row
 * sweep.  Returns the boundary's first entry as (*m, *e) so the work is
 * observable. */
int or_peps_sweep_rows(int L, int W, int D, const double *A, int nrows, int ncols, double *m, int64_t *e) {
    if (nrows < 0 || nrows > L || ncols < 0 || ncols > W || (nrows == L && ncols > 0)) return -1;
    grid_t g = norm_grid(L, W, D, A);
    bnd_t b = bnd_one();
    for (int r = 0; r < nrows; ++r) absorb_row(&g, r, NULL, &b);
    if (ncols > 0) absorb_row_part(&g, nrows, NULL, &b, ncols);
    *m = b.v[0];
    *e = b.e;
    free(b.v);
    grid_free(&g);
    return 0;
}

/* Norm by the plain top-to-bottom row sweep. */
int or_peps_norm(int L, int W, int D, const double *A, double *m, int64_t *e) {
    grid_t g = norm_grid(L, W, D, A);
    bnd_t b = bnd_one();
    for (int r = 0; r < L; ++r) absorb_row(&g, r, NULL, &b);
    *m = b.v[0];
    *e = b.e;
    free(b.v);
    grid_free(&g);
    return 0;
}

static double ratio(double mo, int64_t eo, double mn, int64_t en) {
    return ldexp(mo / mn, (int)(eo - en));
}

/*
 * All observables with cached boundaries.  Outputs (caller-owned):
 *   norm_m, norm_e        the norm as mantissa * 2^exp
 *   sx[L*W]               <X_k> in row-major site order
 *   szsz[nb]              <Z_i Z_j>, horizontal bonds row-major, then vertical
 * Energy is assembled by the caller.
 */
int or_peps_observables(int L, int W, int D, const double *A,
                        double *norm_m, int64_t *norm_e, double *sx, double *szsz) {
    grid_t g = norm_grid(L, W, D, A);
    size_t *off = site_offsets(L, W, D);
    bnd_t *tops = (bnd_t *)malloc(sizeof(bnd_t) * (L + 1));
    bnd_t *bots = (bnd_t *)malloc(sizeof(bnd_t) * (L + 1));
    top_boundaries(&g, tops);
    bottom_boundaries(&g, bots);
    double nm; int64_t ne;
    bnd_dot(&tops[L], &bots[L], &nm, &ne);
    *norm_m = nm; *norm_e = ne;

    double **over = (double **)calloc((size_t)W, sizeof(double *));
    double **ez = (double **)calloc((size_t)L * W, sizeof(double *));
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < W; ++c) {
            int d[4];
            site_dims(L, W, D, r, c, d);
            ez[r * W + c] = double_layer(A + off[r * W + c], d, OP_Z);
        }

    /* sites */
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < W; ++c) {
            int d[4];
            site_dims(L, W, D, r, c, d);
            double *ex = double_layer(A + off[r * W + c], d, OP_X);
            bnd_t b = bnd_copy(&tops[r]);
            over[c] = ex;
            absorb_row(&g, r, over, &b);
            over[c] = NULL;
            double m; int64_t e;
            bnd_dot(&b, &bots[r + 1], &m, &e);
            sx[r * W + c] = ratio(m, e, nm, ne);
            free(b.v); free(ex);
        }
    /* horizontal bonds */
    int k = 0;
    for (int r = 0; r < L; ++r)
        for (int c = 0; c + 1 < W; ++c) {
            bnd_t b = bnd_copy(&tops[r]);
            over[c] = ez[r * W + c]; over[c + 1] = ez[r * W + c + 1];
            absorb_row(&g, r, over, &b);
            over[c] = over[c + 1] = NULL;
            double m; int64_t e;
            bnd_dot(&b, &bots[r + 1], &m, &e);
            szsz[k++] = ratio(m, e, nm, ne);
            free(b.v);
        }
    /* vertical bonds */
    for (int r = 0; r + 1 < L; ++r)
        for (int c = 0; c < W; ++c) {
            bnd_t b = bnd_copy(&tops[r]);
            over[c] = ez[r * W + c];
            absorb_row(&g, r, over, &b);
            over[c] = ez[(r + 1) * W + c];
            absorb_row(&g, r + 1, over, &b);
            over[c] = NULL;
            double m; int64_t e;
            bnd_dot(&b, &bots[r + 2], &m, &e);
            szsz[k++] = ratio(m, e, nm, ne);
            free(b.v);
        }

    for (int q = 0; q < L * W; ++q) free(ez[q]);
    free(ez); free(over);
    for (int r = 0; r <= L; ++r) { free(tops[r].v); free(bots[r].v); }
    free(tops); free(bots); free(off);
    grid_free(&g);
    return 0;
}

/*
 * <Z_k> for every site (Eq. mz with Pauli Z), with cached boundaries:
 * sz[L*W] in row-major site order (caller-owned).  Sec. 3 defines the
 * connected correlator c_ij = <Z_i Z_j> - <Z_i><Z_j> from these and szsz.
 */
int or_peps_sz(int L, int W, int D, const double *A, double *sz) {
    grid_t g = norm_grid(L, W, D, A);
    size_t *off = site_offsets(L, W, D);
    bnd_t *tops = (bnd_t *)malloc(sizeof(bnd_t) * (L + 1));
    bnd_t *bots = (bnd_t *)malloc(sizeof(bnd_t) * (L + 1));
    top_boundaries(&g, tops);
    bottom_boundaries(&g, bots);
    double nm; int64_t ne;
    bnd_dot(&tops[L], &bots[L], &nm, &ne);
    double **over = (double **)calloc((size_t)W, sizeof(double *));
    for (int r = 0; r < L; ++r)
        for (int c = 0; c < W; ++c) {
            int d[4];
            site_dims(L, W, D, r, c, d);
            double *ez = double_layer(A + off[r * W + c], d, OP_Z);
            bnd_t b = bnd_copy(&tops[r]);
            over[c] = ez;
            absorb_row(&g, r, over, &b);
            over[c] = NULL;
            double m; int64_t e;
            bnd_dot(&b, &bots[r + 1], &m, &e);
            sz[r * W + c] = ratio(m, e, nm, ne);
            free(b.v); free(ez);
        }
    free(over);
    for (int r = 0; r <= L; ++r) { free(tops[r].v); free(bots[r].v); }
    free(tops); free(bots); free(off);
    grid_free(&g);
    return 0;
}

/*
 * Nearest-neighbour two-site correlators <A_i B_j> for every bond (i, j) in the
 * output order of szsz (horizontal row-major, then vertical; i the left or
 * upper site), A and B Pauli X (code 1) or Z (code 2), with cached boundaries
 * (Sec. 5: one operator inserted on each of the two sites, then the ratio to
 * the norm).  out[nb] is caller-owned.
 */
int or_peps_bond_ops(int L, int W, int D, const double *A, int op_a, int op_b, double *out) {
    const double *oa = op_a == 1 ? OP_X : OP_Z, *ob = op_b == 1 ? OP_X : OP_Z;
    grid_t g = norm_grid(L, W, D, A);
    size_t *off = site_offsets(L, W, D);
    bnd_t *tops = (bnd_t *)malloc(sizeof(bnd_t) * (L + 1));
    bnd_t *bots = (bnd_t *)malloc(sizeof(bnd_t) * (L + 1));
    top_boundaries(&g, tops);
    bottom_boundaries(&g, bots);
    double nm; int64_t ne;
    bnd_dot(&tops[L], &bots[L], &nm, &ne);
    double **over = (double **)calloc((size_t)W, sizeof(double *));
    int k = 0, d[4];
    for (int r = 0; r < L; ++r)
        for (int c = 0; c + 1 < W; ++c) {
            site_dims(L, W, D, r, c, d);
            double *ea = double_layer(A + off[r * W + c], d, oa);
            site_dims(L, W, D, r, c + 1, d);
            double *eb = double_layer(A + off[r * W + c + 1], d, ob);
            bnd_t b = bnd_copy(&tops[r]);
            over[c] = ea; over[c + 1] = eb;
            absorb_row(&g, r, over, &b);
            over[c] = over[c + 1] = NULL;
            double m; int64_t e;
            bnd_dot(&b, &bots[r + 1], &m, &e);
            out[k++] = ratio(m, e, nm, ne);
            free(b.v); free(ea); free(eb);
        }
    for (int r = 0; r + 1 < L; ++r)
        for (int c = 0; c < W; ++c) {
            site_dims(L, W, D, r, c, d);
            double *ea = double_layer(A + off[r * W + c], d, oa);
            site_dims(L, W, D, r + 1, c, d);
            double *eb = double_layer(A + off[(r + 1) * W + c], d, ob);
            bnd_t b = bnd_copy(&tops[r]);
            over[c] = ea;
            absorb_row(&g, r, over, &b);
            over[c] = eb;
            absorb_row(&g, r + 1, over, &b);
            over[c] = NULL;
            double m; int64_t e;
            bnd_dot(&b, &bots[r + 2], &m, &e);
            out[k++] = ratio(m, e, nm, ne);
            free(b.v); free(ea); free(eb);
        }
    free(over);
    for (int r = 0; r <= L; ++r) { free(tops[r].v); free(bots[r].v); }
    free(tops); free(bots); free(off);
    grid_free(&g);
    return 0;
}

/* E = -J sum <zz> - h sum <x>; also returns everything or_peps_observables does. */
/*
 * <A_i B_j> for any two distinct sites i, j (row-major indices), A and B in
 * {X (1), Z (2), R (4)}: the network with A at site i and B at site j, swept
 * row by row, over the norm swept the same way -- one full contraction per
 * observable, as Sec. 5 counts them.  Returns the ratio in *val.
 */
int or_peps_pair(int L, int W, int D, const double *A, int op_a, int i, int op_b, int j, double *val) {
    if (i == j || i < 0 || j < 0 || i >= L * W || j >= L * W) return -1;
    const double *oa = op_a == 1 ? OP_X : (op_a == 2 ? OP_Z : (op_a == 4 ? OP_R : NULL));
    const double *ob = op_b == 1 ? OP_X : (op_b == 2 ? OP_Z : (op_b == 4 ? OP_R : NULL));
    if (!oa || !ob) return -1;
    grid_t g = norm_grid(L, W, D, A);
    size_t *off = site_offsets(L, W, D);
    int d[4];
    site_dims(L, W, D, i / W, i % W, d);
    double *ea = double_layer(A + off[i], d, oa);
    site_dims(L, W, D, j / W, j % W, d);
    double *eb = double_layer(A + off[j], d, ob);
    double **over = (double **)calloc((size_t)W, sizeof(double *));
    bnd_t n0 = bnd_one(), n1 = bnd_one();
    for (int r = 0; r < L; ++r) {
        absorb_row(&g, r, NULL, &n0);
        over[i % W] = (i / W == r) ? ea : NULL;
        if (j / W == r) over[j % W] = eb;
        absorb_row(&g, r, over, &n1);
        over[i % W] = NULL;
        over[j % W] = NULL;
    }
    *val = ratio(n1.v[0], n1.e, n0.v[0], n0.e);
    free(n0.v); free(n1.v); free(over); free(ea); free(eb); free(off);
    grid_free(&g);
    return 0;
}

/*
 * One observable alone, keeping only two boundaries (for sampled checks of
 * lattices too large for the cached version).  op: 0 = norm (i, j ignored),
 * 1 = X at site i, 2 = Z_i Z_j on the bond (i, j) (site indices, row-major),
 * 3 = Z at site i.
 * Returns the ratio to the norm in *val and the norm in (*nm, *ne).
 */
int or_peps_expect_one(int L, int W, int D, const double *A, int op, int i, int j,
                       double *val, double *nm_out, int64_t *ne_out) {
    grid_t g = norm_grid(L, W, D, A);
    size_t *off = site_offsets(L, W, D);
    int ri = i / W, ci = i % W, rj = j / W, cj = j % W;
    int rlo = 0, rhi = 0;  /* rows [rlo, rhi] carry the insertions */
    if (op == 1 || op == 3) { rlo = rhi = ri; }
    if (op == 2) {
        if (!((ri == rj && cj == ci + 1) || (ci == cj && rj == ri + 1))) {
            free(off); grid_free(&g); return -1;
        }
        rlo = ri; rhi = rj;
    }
    /* top boundary above rlo, bottom boundary below rhi */
    bnd_t top = bnd_one();
    for (int r = 0; r < rlo; ++r) absorb_row(&g, r, NULL, &top);
    grid_t f = grid_flip_rows(&g);
    bnd_t bot = bnd_one();
    for (int r = 0; r < L - 1 - rhi; ++r) absorb_row(&f, r, NULL, &bot);
    grid_free(&f);
    /* norm through the same cut */
    bnd_t nb_ = bnd_copy(&top);
    for (int r = rlo; r <= rhi; ++r) absorb_row(&g, r, NULL, &nb_);
    double nm; int64_t ne;
    bnd_dot(&nb_, &bot, &nm, &ne);
    free(nb_.v);
    *nm_out = nm; *ne_out = ne;
    if (op == 0) { *val = 1.0; goto done; }
    {
        double **over = (double **)calloc((size_t)W, sizeof(double *));
        bnd_t b = bnd_copy(&top);
        int d[4];
        if (op == 1 || op == 3) {
            site_dims(L, W, D, ri, ci, d);
            over[ci] = double_layer(A + off[i], d, op == 1 ? OP_X : OP_Z);
            absorb_row(&g, ri, over, &b);
            free(over[ci]); over[ci] = NULL;
        } else {
            site_dims(L, W, D, ri, ci, d);
            double *zi = double_layer(A + off[i], d, OP_Z);
            site_dims(L, W, D, rj, cj, d);
            double *zj = double_layer(A + off[j], d, OP_Z);
            if (ri == rj) {
                over[ci] = zi; over[cj] = zj;
                absorb_row(&g, ri, over, &b);
            } else {
                over[ci] = zi;
                absorb_row(&g, ri, over, &b);
                over[ci] = NULL; over[cj] = zj;
                absorb_row(&g, rj, over, &b);
            }
            free(zi); free(zj);
        }
        double m; int64_t e;
        bnd_dot(&b, &bot, &m, &e);
        *val = ratio(m, e, nm, ne);
        free(b.v); free(over);
    }
done:
    free(top.v); free(bot.v); free(off);
    grid_free(&g);
    return 0;
}

/* --------------------------------------------- classical Ising (pins) --- */

/*
 * Classical 2D Ising model on the open L x W grid, weight
 * w(s) = prod_<ij> exp(K s_i s_j), enumerated over all 2^N configurations.
 * Outputs Z (as mantissa/exponent relative to exp(K * nb), to avoid overflow),
 * <s_i s_j> per bond (bond order as above) and
 * <exp(-K s_k sum_{j~k} s_j)> per site (the transverse-field expectation of
 * the Ising PEPS, see the tests).  N <= 25.
 */
int or_ising_enumerate(int L, int W, double K, double *logZ, double *corr, double *xflip) {
    int N = L * W;
    if (N > 26) return -1;
    int nb = L * (W - 1) + W * (L - 1);
    int *bi = (int *)malloc(sizeof(int) * nb), *bj = (int *)malloc(sizeof(int) * nb);
    int k = 0;
    for (int r = 0; r < L; ++r) for (int c = 0; c + 1 < W; ++c) { bi[k] = r * W + c; bj[k++] = r * W + c + 1; }
    for (int r = 0; r + 1 < L; ++r) for (int c = 0; c < W; ++c) { bi[k] = r * W + c; bj[k++] = (r + 1) * W + c; }
    uint64_t nconf = 1ull << N;
    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double *zp = (double *)calloc((size_t)nth, sizeof(double));
    double *cp = (double *)calloc((size_t)nth * nb, sizeof(double));
    double *xp = (double *)calloc((size_t)nth * N, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        int s[32];
#pragma omp for schedule(static)
        for (long long cfg = 0; cfg < (long long)nconf; ++cfg) {
            for (int q = 0; q < N; ++q) s[q] = ((cfg >> q) & 1) ? 1 : -1;
            int esum = 0;
            for (int b = 0; b < nb; ++b) esum += s[bi[b]] * s[bj[b]];
            /* weight relative to the all-aligned exp(K nb) */
            double w = exp(K * (double)(esum - nb));
            zp[tid] += w;
            for (int b = 0; b < nb; ++b) cp[(size_t)tid * nb + b] += w * s[bi[b]] * s[bj[b]];
            for (int q = 0; q < N; ++q) {
                int r = q / W, c = q % W, nsum = 0;
                if (r > 0) nsum += s[q - W];
                if (r + 1 < L) nsum += s[q + W];
                if (c > 0) nsum += s[q - 1];
                if (c + 1 < W) nsum += s[q + 1];
                xp[(size_t)tid * N + q] += w * exp(-K * s[q] * nsum);
            }
        }
    }
    double Z = 0.0;
    for (int t = 0; t < nth; ++t) Z += zp[t];
    for (int b = 0; b < nb; ++b) {
        double a = 0.0;
        for (int t = 0; t < nth; ++t) a += cp[(size_t)t * nb + b];
        corr[b] = a / Z;
    }
    for (int q = 0; q < N; ++q) {
        double a = 0.0;
        for (int t = 0; t < nth; ++t) a += xp[(size_t)t * N + q];
        xflip[q] = a / Z;
    }
    *logZ = log(Z) + K * nb;
    free(zp); free(cp); free(xp); free(bi); free(bj);
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
