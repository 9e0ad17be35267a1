/*
 * tn.h -- C-ABI of libtn: exact contraction of open-boundary PEPS on one GB300.
 *
 * What is computed (Sec. 3 of the paper, Eqs. norm, Etot, mx, cij):
 *   <Psi|Psi>, every <X_k> (Eq. mx with S^x = X), every nearest-neighbour
 *   <Z_i Z_j> (first term of Eq. cij) and the transverse-field Ising energy
 *   E = -J sum_<ij> <Z_i Z_j> - h sum_k <X_k> (Eqs. Hamiltonian, Etot), with
 *   Pauli operators (spins +-1) and Z = diag(-1, +1) on the physical index p,
 *   because p = 1 is sigma = +1 (Eq. Psi, x = (sigma + 1)/2); also every
 *   <Z_k> (Eq. mz with Pauli Z) and the connected correlators
 *   c_ij = <Z_i Z_j> - <Z_i><Z_j> (Eq. cij) of the nearest-neighbour bonds.
 *
 * How (Sec. 4): the double-layer network <Psi|O|Psi> (bond dimension D^2) is
 * contracted exactly as chains of pairwise contractions that absorb one site
 * into a large boundary tensor; the lattice is partitioned by the paper's
 * minimum-bottleneck heuristic into up to four corners (row scheme, quadrant
 * scheme or a cut in between) whose ring is closed by dense products.
 *
 * Site tensors (Sec. 5): site (r, c) of an L x W lattice holds
 * A[p][u][l][dn][rt] in C order, p in {0, 1}, bond legs of dimension D and
 * dimension 1 where a leg would leave the lattice (the paper's rank-3 edge and
 * rank-2 corner tensors).  Sites are concatenated in row-major site order, so a
 * lattice has n_elems = sum over sites of 2*u*l*dn*rt FP64 entries (288 for
 * 4x4 D=2, 3872 for 12x12 D=2, 7200 for 8x8 D=3).
 *
 * Outputs: bonds are ordered horizontal (r,c)-(r,c+1) row-major first, then
 * vertical (r,c)-(r+1,c) row-major; nb = L(W-1) + W(L-1).
 *
 * Conventions for every entry point:
 *   - no C++ exception crosses this boundary; every call returns tn_status;
 *   - the caller owns every host buffer passed in; the library copies tensors
 *     on set/submit and owns its device memory, all of which it takes from the
 *     context's HBM budget;
 *   - a handle is used by one host thread at a time, except tn_submit /
 *     tn_poll / tn_wait on one context, which are internally locked;
 *   - a call that needs a GPU returns TN_ERR_NO_DEVICE on a context created
 *     with device = -1 (planning-only context).
 */
#ifndef TN_H
#define TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TN_OK = 0,
    TN_NOT_READY = 1,          /* tn_poll: the job is still running */
    TN_ERR_INVALID = -1,       /* bad argument (sizes, pointers, enum values) */
    TN_ERR_OVER_BUDGET = -2,   /* exact footprint exceeds the context's HBM budget */
    TN_ERR_OOM = -3,           /* device allocation failed inside the budget */
    TN_ERR_CUDA = -4,          /* a CUDA runtime call failed */
    TN_ERR_TIMEOUT = -5,       /* tn_wait deadline passed, or a bounded device wait gave up */
    TN_ERR_NUMERIC = -6,       /* non-finite result or zero norm */
    TN_ERR_NO_DEVICE = -7      /* context has no GPU (device = -1) */
} tn_status;

typedef enum {
    TN_FP64 = 0,      /* FP64 storage and arithmetic */
    TN_FP32 = 1,      /* FP32 storage and arithmetic, FP64 reductions and ratios */
    TN_BF16X3 = 2,    /* FP32 storage; dense ring products on tcgen05 tensor cores,
                         operands split x = x0 + x1 into BF16, 3 products, FP32
                         accumulation (Henry, Tang & Heinecke, ARITH 2019) */
    TN_BF16X6 = 3     /* as TN_BF16X3 with x = x0 + x1 + x2 and 6 products */
} tn_precision;

typedef enum {
    TN_SCHED_AUTO = 0,     /* minimum-bottleneck choice over all cuts (Sec. 4) */
    TN_SCHED_ROW = 1,      /* row scheme, Fig. 2a */
    TN_SCHED_COL = 2,      /* row scheme on the transposed lattice */
    TN_SCHED_QUADRANT = 3  /* quadrant scheme, Fig. 2b, cut at (ceil(L/2), ceil(W/2)) */
} tn_schedule;

typedef enum {
    TN_WORK_NORM = 0,      /* <Psi|Psi> only */
    TN_WORK_ENERGY = 1     /* norm, every <X_k>, every <Z_i Z_j>, every <Z_k> */
} tn_work;

typedef enum {
    TN_OP_NORM = 0,        /* <Psi|Psi> (returned as a ratio 1) */
    TN_OP_X = 1,           /* <X_i>, Eq. mx */
    TN_OP_ZZ = 2,          /* <Z_i Z_j> for nearest neighbours i, j, Eq. cij first term */
    TN_OP_Z = 3,           /* <Z_i>, Eq. mz with Pauli Z */
    TN_OP_Y = 4            /* <Y_i>, Pauli Y = [[0, i], [-i, 0]] on p = 0, 1 (sigma_y with
                              rows and columns in the order sigma = -1, +1).  For real
                              site tensors Y = i R with the real R = [[0, 1], [-1, 0]],
                              so <Y_i> = <A_i Y_j> = 0 (A = X, Z) exactly and
                              <Y_i Y_j> = -<R_i R_j>; complex site tensors contract Y */
} tn_op;

/* value = mant * 2^exp2 (the norm of a large lattice leaves the FP64 range). */
typedef struct {
    double mant;
    int64_t exp2;
} tn_scalar;

typedef struct {
    double energy;            /* E for the (J, h) of the call */
    double energy_per_site;   /* E / (L W) */
    tn_scalar norm;           /* <Psi|Psi> */
    double *sx;               /* caller-owned, L*W entries, or NULL */
    double *szsz;             /* caller-owned, nb entries, or NULL */
    double err_bound_est;     /* a-priori relative rounding bound of the precision used */
    int precision;            /* tn_precision used */
    int schedule_o, schedule_i, schedule_j;   /* partition actually used (see tn_plan) */
    double *sz;               /* caller-owned, L*W entries <Z_k>, or NULL */
    double *czz;              /* caller-owned, nb entries c_ij = <Z_i Z_j> - <Z_i><Z_j>, or NULL */
} tn_result;

typedef struct tn_ctx tn_ctx;
typedef struct tn_lattice tn_lattice;
typedef struct tn_batch tn_batch;
typedef struct tn_batch_group tn_batch_group;

/* ----------------------------------------------------------- context ---- */

/* Create a context on CUDA device `device` (or -1: planning only, no GPU).
 * hbm_budget_bytes caps every device allocation the library makes (0 = 90% of
 * the device's free memory).  cuda_stream (a cudaStream_t, or NULL for a
 * stream the context creates) is where every kernel of this context runs. */
tn_status tn_ctx_create(int device, size_t hbm_budget_bytes, void *cuda_stream, tn_ctx **out);
tn_status tn_ctx_destroy(tn_ctx *ctx);
/* Bytes of the budget currently held by lattices, batches and jobs. */
tn_status tn_ctx_memory(const tn_ctx *ctx, size_t *used, size_t *budget);

/* ----------------------------------------------------------- lattices --- */

/* A lattice of L x W sites, bond D (1 <= L, W <= 16, 1 <= D <= 4).  Tensors
 * start at zero.  Works on a planning-only context (no device memory). */
tn_status tn_create_lattice(tn_ctx *ctx, int L, int W, int D, tn_lattice **out);
tn_status tn_destroy_lattice(tn_lattice *lat);
/* Number of FP64 entries the site tensors of (L, W, D) take (layout above). */
size_t tn_lattice_elems(int L, int W, int D);
/* Copy n_elems host doubles (must equal tn_lattice_elems) into the lattice. */
tn_status tn_set_site_tensors(tn_lattice *lat, const double *host, size_t n_elems);
/* Fill with i.i.d. uniform[-1,1) from `seed`: SplitMix64 (Steele, Lea & Flood
 * 2014) as a counter-based generator, entry k (fill order above) is
 * 2 * (mix64(seed + (k+1) * 0x9E3779B97F4A7C15) >> 11) * 2^-53 - 1. */
tn_status tn_fill_random(tn_lattice *lat, uint64_t seed);
/* Copy the lattice's FP64 tensors back to the host (n_elems entries);
 * TN_ERR_INVALID for a lattice holding complex tensors. */
tn_status tn_get_site_tensors(const tn_lattice *lat, double *host, size_t n_elems);
/* Complex site tensors A = re + i im (Eq. Psi with complex amplitudes), each
 * array n_elems doubles in the layout above.  Every later contraction of the
 * lattice (norm, expectations, energy, bond and pair correlators, <Y_k>)
 * uses the double layer sum_{p,q} conj(A_p) O_pq A_q (Sec. 5, bra layer
 * conjugated), built in a real basis of Hermitian matrices per bond so that
 * every contraction after the site matrices stays real arithmetic.
 * tn_set_site_tensors / tn_fill_random return the lattice to real tensors.
 * Served jobs, batches, the boundary MPS and the imaginary time evolution
 * take real tensors only. */
tn_status tn_set_site_tensors_complex(tn_lattice *lat, const double *re, const double *im, size_t n_elems);
/* 1 if the lattice holds complex site tensors, else 0. */
int tn_lattice_is_complex(const tn_lattice *lat);

/* ------------------------------------------------------------ planning -- */

/* Exact device bytes the library allocates to run `work` on this lattice with
 * this schedule and precision (the arena admission control checks), for the
 * program choices the tuning table holds for the shape (see tn_autotune):
 * with bit 5 set, the recompute form's bytes. */
tn_status tn_footprint(const tn_lattice *lat, tn_schedule sched, tn_precision prec,
                       tn_work work, size_t *peak_bytes);
/* The contraction schedule chosen by the heuristic of Sec. 4 as int64 words:
 *   [0] = 1 (format), [1] = o, [2] = i, [3] = j, [4] = number of steps,
 *   [5] = bottleneck entries, [6] = multiply-adds of one norm,
 *   then 9 words per site-absorption step:
 *   corner (0 TL, 1 TR, 2 BL, 3 BR), frame row k, frame column c,
 *   lattice row r, lattice column c, P, K, N, S
 * where the step maps the boundary [P, K, S] to [P, N, S].  o = 1 means the
 * cut (i, j) is taken on the transposed lattice.  Writes at most cap words
 * and the full length to *n. */
tn_status tn_plan(const tn_lattice *lat, tn_schedule sched, int64_t *out, size_t cap, size_t *n);
/* As tn_plan for a given work.  TN_WORK_NORM is tn_plan.  TN_WORK_ENERGY keeps
 * every chain state for its environment sweeps, so among the cuts with the
 * smallest bottleneck it prefers the smallest summed chain output, then the
 * fewest multiply-adds (word [6] is still the norm's multiply-adds). */
tn_status tn_plan_work(const tn_lattice *lat, tn_schedule sched, tn_work work, int64_t *out, size_t cap,
                       size_t *n);

/* Contraction program of the lattice (host only, no device needed): builds it
 * as a contraction would and checks it -- every pairwise contraction runs
 * after the contractions producing its inputs and within their lifetimes, and
 * no two tensors alive at the same time share memory (TN_ERR_NUMERIC with the
 * reason in tn_last_error otherwise).  Writes at most cap words to out and the
 * full length to *n:
 *   [0] contractions (ops)   [1] waves   [2] arena bytes   [3] footprint bytes
 *   [4] absorption-family algorithmic bytes (single steps, fused step pairs
 *       and absorb-dots)      [5] fused step pairs   [6] product multiply-adds
 * work: TN_WORK_NORM or TN_WORK_ENERGY. */
tn_status tn_program_info(const tn_lattice *lat, tn_precision prec, tn_schedule sched, tn_work work,
                          int64_t *out, size_t cap, size_t *n);

/* ---------------------------------------------------------- contraction -- */

/* <Psi|Psi> (blocking). */
tn_status tn_contract_norm(tn_lattice *lat, tn_precision prec, tn_schedule sched, tn_scalar *out);
/* One expectation value (blocking): op = TN_OP_X, TN_OP_Y or TN_OP_Z with
 * site i = r*W + c, or TN_OP_ZZ with nearest-neighbour sites i < j.  Returns
 * the ratio to the norm. */
tn_status tn_expectation(tn_lattice *lat, tn_precision prec, int op, int i, int j, double *out);
/* <O_k> for every site k (row-major), O = TN_OP_X, TN_OP_Y or TN_OP_Z
 * (Eqs. mx, mz; blocking, AUTO schedule).  out: L*W doubles, caller-owned. */
tn_status tn_site_expectations(tn_lattice *lat, tn_precision prec, int op, double *out);
/* Norm, every <X_k>, every <Z_i Z_j>, every <Z_k>, the connected c_ij and E
 * for (J, h) (blocking, AUTO schedule); each array of *out is filled if non-NULL.
 * When the program with every chain state cached does not fit the context's
 * budget left, this call and every other observable call on the lattice
 * (tn_expectation, tn_site_expectations, tn_bond_correlators,
 * tn_pair_correlators) take the recompute form (program choice bit 5: the
 * same values, bit for bit, in less memory); TN_ERR_OVER_BUDGET if that does
 * not fit either.  Served jobs do not fall back (tn_submit). */
tn_status tn_energy(tn_lattice *lat, double J, double h, tn_precision prec, tn_result *out);
/* Nearest-neighbour two-site correlators <A_i B_j> (blocking, AUTO schedule):
 * one Pauli operator on each site of every bond, A = op_a on the bond's first
 * site i (left or upper) and B = op_b on j, op_a and op_b each TN_OP_X,
 * TN_OP_Y or TN_OP_Z (the insertion of Sec. 5 with operators other than Z Z;
 * Y as described at TN_OP_Y).  out: nb = L(W-1) + W(L-1) doubles,
 * caller-owned, bonds in the order of tn_result.szsz.  TN_ERR_INVALID for
 * other operators. */
tn_status tn_bond_correlators(tn_lattice *lat, tn_precision prec, int op_a, int op_b, double *out);
/* <A_{i[k]} B_{j[k]}> for n arbitrary pairs of distinct sites (row-major
 * indices; Eq. cij for any i, j), A = op_a, B = op_b in {TN_OP_X, TN_OP_Y,
 * TN_OP_Z}, exactly (blocking, AUTO schedule).  The contraction program is
 * built for the call: pairs inside one corner carry the chain from the first
 * site to the second and meet that corner's environment; pairs in two corners
 * regrow both and close the ring by one product (adjacent corners) or two
 * (diagonal corners).  out: n doubles, caller-owned.  TN_ERR_INVALID for bad
 * sites or operators. */
tn_status tn_pair_correlators(tn_lattice *lat, tn_precision prec, int op_a, int op_b, int n, const int *i,
                              const int *j, double *out);
/* As tn_energy with an explicit schedule. */
tn_status tn_energy_sched(tn_lattice *lat, double J, double h, tn_precision prec,
                          tn_schedule sched, tn_result *out);

/* ------------------------------------------------------------- batches --- */

/* n independent lattices of possibly different (L, W, D), evaluated together:
 * every wave of site absorptions and dense products of all members runs as one
 * grouped launch; the launch sequence is captured once into a CUDA graph and
 * replayed.  Device memory for all members is taken from the budget here. */
tn_status tn_batch_create(tn_ctx *ctx, int n, const int *L, const int *W, const int *D,
                          tn_precision prec, tn_schedule sched, tn_work work, tn_batch **out);
tn_status tn_batch_destroy(tn_batch *b);
/* Total FP64 entries of all members' tensors (members in order). */
size_t tn_batch_elems(const tn_batch *b);
/* Member tensors, concatenated in member order: from host memory, from device
 * memory (a device pointer), or from the generator (member k uses seed
 * mix64(batch_seed + (k+1) * 0x9E3779B97F4A7C15)).  Asynchronous on the ctx
 * stream; the host buffer must stay valid until the next synchronising call. */
tn_status tn_batch_set_tensors(tn_batch *b, const double *host, size_t n_elems);
tn_status tn_batch_set_tensors_device(tn_batch *b, const double *dev, size_t n_elems);
tn_status tn_batch_fill_random(tn_batch *b, uint64_t batch_seed);
/* Run the whole batch (asynchronous on the ctx stream).  h holds one field per
 * member; J is shared. */
tn_status tn_batch_run(tn_batch *b, double J, const double *h);
/* Per member: 6 + 2 L*W + nb doubles [energy, log2 norm, norm mantissa, norm
 * exponent, sum_k <X_k>, sum_<ij> <Z_i Z_j>, <X_k>..., <Z_i Z_j>..., <Z_k>...]
 * (work = ENERGY) or 6 doubles (NORM), members concatenated.  E at any other
 * field is -J * [5] - h * [4].  _size gives the total; _host synchronises and copies;
 * _device returns the device pointer of the same array (valid until the next
 * run). */
size_t tn_batch_result_size(const tn_batch *b);
tn_status tn_batch_results_host(tn_batch *b, double *host, size_t cap);
tn_status tn_batch_results_device(tn_batch *b, const double **dev);
/* Number of kernel launches one tn_batch_run issues. */
tn_status tn_batch_launch_count(const tn_batch *b, int64_t *n);

/* Batch groups (no counterpart in the paper; many lattices of uneven sizes
 * in one launch): n lattices whose summed footprint may exceed the
 * device.  Members are split, in order, into passes of at most pass_budget
 * bytes each; the passes run one after another and share one arena (the
 * largest pass's), each keeping its small regions (inputs, slots, results,
 * tables); the launches of all passes are captured into ONE CUDA graph, so a
 * run of the whole group is one graph launch.  A member whose energy program
 * alone exceeds pass_budget with its chain states cached takes the recompute
 * form (program choice bit 5) when that fits.  TN_ERR_OVER_BUDGET when a
 * member alone still exceeds pass_budget or the arena the remaining budget;
 * TN_ERR_NO_DEVICE without a device.  Inputs and results are concatenated in
 * member order with the layouts of tn_batch_*; member k of the generator
 * takes the seed member k of one batch would. */
tn_status tn_batch_group_create(tn_ctx *ctx, int n, const int *L, const int *W, const int *D,
                                tn_precision prec, tn_schedule sched, tn_work work, size_t pass_budget,
                                tn_batch_group **out);
tn_status tn_batch_group_destroy(tn_batch_group *g);
/* Passes, shared arena bytes, total input entries, total result doubles and
 * kernel launches per run (any pointer may be NULL). */
tn_status tn_batch_group_info(const tn_batch_group *g, int *passes, size_t *arena_bytes, size_t *n_elems,
                              size_t *n_results, int64_t *launches);
tn_status tn_batch_group_set_tensors(tn_batch_group *g, const double *host, size_t n_elems);
tn_status tn_batch_group_fill_random(tn_batch_group *g, uint64_t batch_seed);
/* One graph launch for every member (asynchronous on the ctx stream). */
tn_status tn_batch_group_run(tn_batch_group *g, double J, const double *h);
tn_status tn_batch_group_results_host(tn_batch_group *g, double *host, size_t cap);

/* ------------------------------------------------------------- serving --- */

typedef struct {
    int L, W, D;
    tn_precision precision;
    double J, h;
    const double *tensors;   /* host, tn_lattice_elems(L,W,D) entries, copied at submit; or NULL */
    uint64_t seed;           /* used when tensors == NULL (tn_fill_random's generator) */
} tn_job;

/* Queue a job.  It is admitted to the GPU when its exact footprint fits the
 * budget left by running jobs; jobs that can never fit return
 * TN_ERR_OVER_BUDGET here.  Jobs take the tuning table's program choices and
 * do not fall back to the recompute form: a job whose cached-state program
 * exceeds the budget would hold the device for seconds to minutes, which a
 * latency-bound stream refuses instead (set bit 5 for the shape by hand to
 * serve it).  Admitted jobs run concurrently with earlier ones:
 * jobs whose estimated device time (from their contraction program) is at
 * most 20 ms are batched together on high-priority streams, longer ones run
 * alone on low-priority streams, so short jobs never queue behind long ones. */
tn_status tn_submit(tn_ctx *ctx, const tn_job *job, uint64_t *ticket);
/* TN_NOT_READY until the job is done; then fills *out (sx/szsz if non-NULL)
 * and releases the ticket. */
tn_status tn_poll(tn_ctx *ctx, uint64_t ticket, tn_result *out);
/* As tn_poll but blocks up to timeout_s seconds (TN_ERR_TIMEOUT after). */
tn_status tn_wait(tn_ctx *ctx, uint64_t ticket, double timeout_s, tn_result *out);

/* -------------------------------------------------- kernel entry points -- */

/* One site absorption on device buffers (the pairwise contraction of Sec. 4
 * that dominates the paper's profile, Sec. 7):
 *   out[p][n][s] = sum_k in[p][k][s] * E[k][n],  p < P, k < K, n < N, s < S,
 * all arrays C order, dtype 0 = FP64, 1 = FP32.  Runs on `stream`; no
 * rescaling.  Returns TN_ERR_INVALID for non-positive sizes or NULL pointers. */
tn_status tn_absorb(int dtype, const void *in, const void *E, void *out,
                    int64_t P, int32_t K, int32_t N, int64_t S, void *stream);

/* The same absorption fused with a dot product against a tensor of the output
 * shape -- the last step of every observable of Sec. 5, where the state with
 * an operator inserted meets its environment:
 *   *result = sum_{p,n,s} (sum_k in[p][k][s] E[k][n]) * adj[p][n][s]
 * in, E, adj: device arrays of dtype 0 = FP64 / 1 = FP32 (C order, shapes as
 * tn_absorb, adj [P][N][S]); result: device pointer to one double.  Each tile
 * of 256 outer positions adds its products into one FP64 partial; the last
 * tile sums the partials in index order, so the result is bit-reproducible.
 * The partials (8 bytes per tile, plus a 16-byte counter) are scratch the call
 * takes with cudaMallocAsync on `stream` and returns with cudaFreeAsync.
 * Returns TN_ERR_INVALID for bad sizes or NULL pointers, TN_ERR_OOM if the
 * scratch cannot be allocated. */
tn_status tn_absorb_dot(int dtype, const void *in, const void *E, const void *adj,
                        int64_t P, int32_t K, int32_t N, int64_t S, double *result, void *stream);

/* tn_absorb_dot without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not call the CUDA allocator
 * where they call us -- a latency-critical loop (cudaMalloc / cudaFree may
 * synchronise the whole device), or a process whose device memory is already
 * held by another allocator, so a new allocation could fail.  Arguments,
 * result and errors are those of tn_absorb_dot; the caller still owns every
 * input and the output.
 *   Scratch: one fixed array of 16 + 8 * 65536 bytes (about 512 KiB) compiled
 *   into the library; every GPU that loads libtn holds it until the process
 *   exits.  Its size caps the problem: P * S <= 16,777,216 (65,536 tiles of
 *   256 outer positions); larger calls return TN_ERR_INVALID without touching
 *   the GPU.
 *   Set-up: the first call on a device (the calling thread's current device,
 *   which `stream` must belong to) looks up the array's device address; make
 *   that first call before any stream capture.
 *   Sharing: every call on a device uses the same array and the array keeps
 *   the last call's contents; each call clears the part that must start at
 *   zero.  Calls whose executions overlap on the GPU (different streams, no
 *   ordering between them) race on the array and give wrong results. */
tn_status tn_absorb_dot_noalloc(int dtype, const void *in, const void *E, const void *adj,
                                int64_t P, int32_t K, int32_t N, int64_t S, double *result,
                                void *stream);

/* ------------------------------------------- imaginary time evolution --- */

/* Parameters of an imaginary time evolution (Sec. 5): H = -J sum_<ij> Z_i Z_j
 * - gamma sum_k X_k, steps of U(dtau) = U^Gamma(dtau/2) U^J(dtau) U^Gamma(dtau/2)
 * (second-order Trotter-Suzuki).  A two-site update keeps the singular values
 * with lambda_k / lambda_1 >= eps (Sec. 6), at most chi_max of them; chi_max
 * must equal the lattice's bond dimension D, which is the storage dimension
 * of every bond (bonds with fewer kept values are zero-padded, which leaves
 * the state unchanged).  energy_every > 0 evaluates E by the exact
 * contraction, in `precision`, after every energy_every-th step. */
typedef struct {
    double J, gamma, dtau;
    int steps;
    int chi_max;
    double eps;
    int energy_every;
    int precision;        /* tn_precision of the energy evaluations */
} tn_ite_params;

/* Set the lattice to the initial state of Sec. 5, the uniform superposition
 * prod_k (|+1> + |-1>) / sqrt 2: every site A[p][0][0][0][0] = 1/sqrt 2, all
 * other entries (the padding of bonds of dimension 1) zero. */
tn_status tn_ite_init_product(tn_lattice *lat);
/* Evolve the lattice's state in place on the GPU (Sec. 5, Fig. 3):
 * per step, the one-body gates exp(gamma dtau/2 X) on every site, then the
 * two-body gates exp(J dtau Z_i Z_j) on every bond in four classes of disjoint
 * bonds (horizontal bonds whose left site has an even column, then odd;
 * vertical bonds whose upper site has an even row, then odd) -- each bond's
 * gate contracted with its two sites, the result matricised (rows: the first
 * site's physical index and other legs, columns: the second site's) and split
 * by an FP64 one-sided Jacobi SVD into U sqrt(lambda) and sqrt(lambda) V^T --
 * then the one-body gates again; after each of the three sets the state is
 * divided by sqrt(<Psi|Psi>), the norm contracted exactly in FP64.
 * energies: steps / energy_every doubles (caller-owned) or NULL; bond_dims:
 * nb ints, the number of singular values each bond kept at its last update
 * (bond order of tn_result.szsz), or NULL; max_discarded: the largest
 * lambda_k / lambda_1 any truncation dropped, or NULL.  The lattice's host
 * tensors hold the evolved state on return.  Device memory for the program
 * buffers and an SVD workspace (m n + n^2 doubles per bond of a class, m, n
 * <= 2 D^3) comes from the context's budget.  TN_ERR_INVALID for bad
 * parameters, TN_ERR_NUMERIC for a non-finite energy. */
tn_status tn_ite_run(tn_lattice *lat, const tn_ite_params *params, double *energies, int *bond_dims,
                     double *max_discarded);

/* ------------------------------------------------------------ autotuner -- */

/* Program choices per lattice shape (no counterpart in the paper; the tuned
 * tiles and schedules of the batched form).  Each choice is an exact
 * reformulation -- only speed differs:
 *   bit 0  FP32 D = 2: two steps of a frame row fused in one pass
 *   bit 1  FP32 D <= 2: <X_k>, <Z_k> and the local norm in one absorb-dot
 *   bit 2  D = 3 interior steps: ket pass then bra pass on FP32 / FP64 ALUs
 *          (cleared: the double-layer site matrix, absorbed on the tensor
 *          cores in BF16x3 / BF16x6)
 *   bit 3  BF16x3 / BF16x6: products of at least 2^26 multiply-adds on the
 *          tensor cores (else FP32 SIMT)
 *   bit 4  BF16x3 / BF16x6: smaller products on the tensor cores too
 *   bit 5  energies and correlators: the recompute form -- the corner chains
 *          keep only the states that start a frame row (and the finished
 *          corners); each observable absorbs the states it needs again from
 *          the checkpoint before them, and the environment sweep of Sec. 5
 *          holds one state at a time, corner after corner.  The same
 *          contractions on the same inputs, so the same bits, in a fraction of
 *          the memory (10 x 10, D = 3, FP32: 155 GB instead of 692 GB) for
 *          more absorptions; never chosen by tn_autotune, set by hand or taken
 *          as the fallback described at tn_energy
 * 15 (bits 0-3 set) is the fixed default; codes run from 0 to 63.  tn_autotune times every combination that
 * changes the program of each distinct (L[k], W[k], D[k]) on a batch of
 * copies of it (as many as fit max_bytes, 0 = 4 GiB, at most 64; shapes whose
 * single footprint exceeds max_bytes are skipped), `reps` timed runs after one
 * warm-up, CUDA events on the batch's stream, and stores the fastest (a
 * combination replaces the current choice only when 2% faster) in a process-
 * wide table keyed on (L, W, D, precision, work).  Batches, lattices and served
 * jobs created afterwards use the table's choice for their shape, so a lattice
 * is contracted the same way alone, in a batch and when served; tune before
 * creating them.  work: TN_WORK_NORM or TN_WORK_ENERGY. */
tn_status tn_autotune(tn_ctx *ctx, int n, const int *L, const int *W, const int *D, tn_precision prec,
                      tn_work work, int reps, size_t max_bytes);
/* The table's choice for a shape: knobs (15 if untuned), the tuned and the
 * default mean ms per batch run of the tuning batch, tuned = 1 if present. */
tn_status tn_autotune_lookup(int L, int W, int D, tn_precision prec, tn_work work, int *knobs, double *best_ms,
                             double *default_ms, int *tuned);
/* Set a shape's choice by hand (knobs 0..63; TN_ERR_INVALID otherwise). */
tn_status tn_autotune_set(int L, int W, int D, tn_precision prec, tn_work work, int knobs);
tn_status tn_autotune_clear(void);
/* The table as text, one shape per line; load merges a saved table. */
tn_status tn_autotune_save(const char *path);
tn_status tn_autotune_load(const char *path);

/* -------------------------------------- boundary-MPS approximate contraction */

/* Approximate contraction of the double-layer network by a boundary MPS of
 * bond chi -- the environment approximation the paper names as the way past
 * the exact method's memory limit (Sec. 7).  The top row is a matrix product
 * state whose physical legs are the rows' down legs; each further row is
 * applied as a matrix product operator and the result compressed back to bond
 * chi (right-orthonormalised right to left, then cut by SVD left to right,
 * keeping the chi largest singular values; one-sided Jacobi SVDs).  With
 * chi >= (D^2)^floor(W/2) nothing is dropped and the result is exact.
 * prec: TN_FP64, or TN_FP32 (every tensor and SVD in FP32: the truncation
 * error of an approximate contraction is far above FP32 rounding, and the
 * GB300 runs FP32 at 64 times its FP64 rate; singular values below 3e-6 of the
 * largest are dropped as zero); other precisions return TN_ERR_INVALID.
 * chi must satisfy max(chi, D^2) * D^2 <= 512.  Every network is contracted by
 * one block of one launch, its workspace (about (2W + 2) B^2 D^2 + B^2 + D^8
 * doubles, B = max(chi, D^2) D^2) taken from the context's budget for the call.
 * tn_bmps_norm: <Psi|Psi>. */
tn_status tn_bmps_norm(tn_lattice *lat, int chi, tn_precision prec, tn_scalar *out);
/* <A_i> (op_j = 0) or <A_i B_j> (i != j) for A, B in {TN_OP_X, TN_OP_Z}, any
 * sites: the network with the operators inserted over the norm, both by the
 * boundary MPS (two networks, one launch). */
tn_status tn_bmps_expectation(tn_lattice *lat, int chi, tn_precision prec, int op_i, int i, int op_j, int j,
                               double *out);
/* The norm, every <X_k> and every nearest-neighbour <Z_i Z_j> (1 + N + nb
 * networks in one launch, Sec. 5's one contraction per observable, each by the
 * boundary MPS), and E = -J sum <ZZ> - h sum <X>; out->sx / out->szsz filled if
 * non-NULL; out->sz and out->czz untouched. */
tn_status tn_bmps_energy(tn_lattice *lat, int chi, tn_precision prec, double J, double h, tn_result *out);

/* ------------------------------------------------------------ misc -------- */

const char *tn_status_string(tn_status s);
/* Message of the last failing call on this host thread ("" if none). */
const char *tn_last_error(void);
/* Bounded-wait self-check (no counterpart in the paper; failure detection of
 * the library's device waits): launches one thread that waits on a device flag
 * nothing sets, bounded by limit_ms of GPU clock, as every pipelined kernel's
 * wait is; *expired receives 1 when the wait ran out and the kernel exited
 * cleanly (the context stays usable), 0 otherwise.  Allocates 8 bytes of
 * device memory for the call.  TN_ERR_INVALID for limit_ms outside (0, 10000]. */
tn_status tn_wait_selfcheck(tn_ctx *ctx, double limit_ms, int *expired);
/* Measured FMA rate of the context's device in TFLOP/s (no counterpart in the
 * paper; the denominator of the ALU-bound roofline figures): dtype 0 = FP64
 * fma, 1 = FP32 fma.rn.f32x2, 8 independent chains per thread, 2048 threads
 * per SM, best of three launches timed with CUDA events on the context's
 * stream.  Allocates 16 bytes of device memory for the call. */
tn_status tn_peak_probe(tn_ctx *ctx, int dtype, double *tflops);
/* Host-side fault injection (no counterpart in the paper; failure detection):
 * the next `count` batch runs of this context -- served batches, tn_energy and
 * the other blocking calls, tn_batch_run -- have their status word set after
 * their kernels are queued, exactly as a bounded device wait that ran out
 * would set it, so the error path (TN_ERR_TIMEOUT from tn_poll / tn_wait, the
 * blocking calls and tn_batch_results_host) can be tested without disturbing
 * any kernel.  count = 0 disarms.  TN_ERR_INVALID for count < 0. */
tn_status tn_ctx_inject_wait_timeout(tn_ctx *ctx, int count);
/* Per kernel family since the last reset: launches, summed device time (ms,
 * from CUDA events around each launch, only while profiling is on),
 * algorithmic bytes and multiply-adds.  family: 0 absorb (one step),
 * 1 absorb-dot (one step, with one to three site matrices), 2 SIMT dense
 * product, 3 tensor-core dense product, 4 other, 5 two steps of a frame row
 * fused (with or without the final dot). */
tn_status tn_ctx_set_profiling(tn_ctx *ctx, int on);
tn_status tn_ctx_kernel_stats(tn_ctx *ctx, int family, int64_t *launches, double *ms,
                              double *bytes, double *macs);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */
