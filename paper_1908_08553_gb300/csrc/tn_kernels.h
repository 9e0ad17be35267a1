// Plain-old-data task descriptors shared by the host executor and the CUDA
// kernels, and the host-side launch wrappers.  Every kernel processes a list of
// independent tasks (all members of a batch, all corners, all observables of a
// wave) in one launch; a block finds its task by a binary search over the
// tasks' first tile index.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace tn {

// Per-tensor bookkeeping of the power-of-two rescaling.  A tensor's true value
// is stored * 2^X.  maxbits collects max|stored| (as FP64 bits, atomicMax) while
// the tensor is produced; a consumer multiplies every loaded entry by 2^-e with
// e = frexp exponent of that max, so its inputs are in [-1, 1).  Scalar results
// keep their FP64 mantissa in `mant`; `count` orders the deterministic final
// reduction of per-tile partial sums.
struct Slot {
    long long X;
    unsigned long long maxbits;
    double mant;
    unsigned int count;
    unsigned int pad;
};
static_assert(sizeof(Slot) == 32, "slot layout");

struct AbsorbTask {
    const void* in;
    const void* E;
    void* out;            // unused in dot mode
    const void* adj;      // dot mode: adjoint tensor [P][N][S]
    double* partial;      // dot mode: one FP64 partial per tile
    unsigned* counter;    // plain dot mode: tile arrival counter (zeroed before launch)
    long long P, S;
    long long tile0;      // first global tile of this task
    int K, N;
    int transE;           // 1: use E[n][k] as E[k][n] (backward / environment sweep)
    int slot_in, slot_E, slot_out, slot_adj;
    int ntiles;
    // dual / triple dot modes: a second (third) site matrix on the same input
    // and adjoint, its result in slot_out2 (slot_out3); partials of the k-th
    // result at k * ntiles
    const void* E2;
    const void* E3;
    int slot_E2, slot_out2, slot_E3, slot_out3;
};

struct GemmTask {
    // C[m][n] = sum_k A(m,k) B(k,n), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]
    const void* A;
    const void* B;
    void* C;              // row-major [M][N]; unused in dot mode
    const void* Dm;       // dot mode: partner, row-major [M][N]
    double* partial;
    long long M, N, K;
    long long sam, sak, sbk, sbn;
    long long tile0;
    long long kslice;     // k per tile (= K unless the product is split along k)
    int tiles_n, ntiles;
    int ksplit;           // tiles along k (dot mode: one FP64 partial each)
    int slot_A, slot_B, slot_C, slot_D;
};

// k-slice of the products fused with a dot: partial sums of at most this
// many FP32 terms before the FP64 accumulation.
constexpr long long kGemmKSlice = 512;

struct DotTask {
    const void* A;
    const void* B;
    double* partial;
    long long n;
    long long tile0;
    int ntiles;
    int slot_A, slot_B, slot_out;
};

struct SiteMatTask {
    const double* A;      // raw FP64 site tensor [p][u][l][dn][rt]
    const double* Ai;     // its imaginary parts (complex site tensors), else null
    void* E;              // K x N, compute dtype
    int dims[4];          // original leg dims u, l, dn, rt
    int map[4];           // frame role (u, l, dn, rt) -> original leg
    int phys;             // 0 I, 1 X, 2 Z, 3 R, 4 Y (complex only)
    int slot_E;
    int K, N;
    int factored;         // 1: the two layer factors of the double-layer matrix (kFactorEntries)
};

// Interior D = 3 steps (K = N = 81, every frame leg of dimension 3) keep the
// double-layer site matrix as its two layer factors, 2 x 9 x 9 entries each:
//   Fa[p][(h u)][(dn rt)] = A[p](frame legs of layer a) 2^-e_A
//   Fb[p][(h u)][(dn rt)] = sum_q O[p][q] A[q](frame legs of layer b) 2^-e_A
// so that E[(h_a h_b)(u_a u_b)][(dn_a dn_b)(rt_a rt_b)] = sum_p Fa Fb.
constexpr int kFactorEntries = 4 * 81;

// Result header per member: E, log2 norm, norm mantissa, norm exponent,
// sum <X>, sum <ZZ>; then <X_k> and <Z_i Z_j>.
constexpr int kResultHeader = 6;

struct FinalTask {
    const int* sx_slots;  // n_sites
    const int* zz_slots;  // n_bonds
    const int* sx_den;    // n_sites: slot of each ratio's denominator
    const int* zz_den;    // n_bonds
    const int* sz_slots;  // n_sites: <Z_k> numerators (same denominators as sx)
    const int* sy_slots;  // n_sy (0 or n_sites): <Y_k> numerators (complex site tensors)
    double* out;          // kResultHeader + 2 n_sites + n_bonds + n_sy: <X_k>, <Z_i Z_j>, <Z_k>, <Y_k>
    double J, h;
    int norm_slot;
    int n_sites, n_bonds, n_sy;
};

struct ConstOne {
    void* ptr;
};

// FP32 operand X[r][k] = src[r*sr + k*sk] (rescaled by its slot) split into
// BF16 planes in the tiled tensor-core layout (see tc_gemm.cu).
struct TcSplitTask {
    const void* src;
    void* dst;
    long long R, Kd, sr, sk;      // logical rows, reduction length, strides
    long long Rp, Kp;             // padded to 128 rows, 64 k
    long long plane_bytes;
    long long tile0;
    int ntiles, nsplit, slot_src, pad;
};

// C[m][n] = sum_k A[m][k] B[n][k] from tiled BF16 planes, 128 x 128 tiles.
struct TcGemmTask {
    const void* A;                // tiled planes of A (rows m)
    const void* B;                // tiled planes of B (rows n)
    void* C;                      // FP32 [M][N] (store mode)
    const void* Dm;               // FP32 [M][N] dot partner (dot mode)
    double* partial;
    long long a_plane_bytes, b_plane_bytes;
    long long M, N, Kp;
    long long tile0;
    long long kchunks;            // 64-wide k chunks per tile (split along k in dot mode)
    long long tiles_m;
    int tiles_n, ntiles;
    int ksplit;
    int slot_A, slot_B, slot_C, slot_D;   // slots of the FP32 sources / result
};

// One bond of an imaginary-time two-body update (Sec. 5, Fig. 3): sites i and j
// (offsets in FP64 entries into the site array, dims {2, u, l, dn, rt}), the
// bond between them (i's rt and j's l when horizontal, i's dn and j's u when
// vertical), Theta of m x n (rows: i's p and other legs, columns: j's), and a
// workspace of m * n2 + n2 * n2 doubles (n2 = n rounded up to even).
struct IteBondTask {
    long long off_i, off_j, ws_off;
    int dims_i[5], dims_j[5];
    int horizontal;
    int m, n;
};

// One network of a boundary-MPS contraction (bmps.cu): the double-layer norm
// network of an L x W PEPS of bond D (FP64 site tensors in the input layout),
// with up to two Pauli operators inserted (code 1 X, 2 Z at op_site; -1: none),
// contracted with boundary bond chi; out receives (mantissa, exponent).
struct BmpsTask {
    const double* A;
    double* ws;
    double* out;
    int L, W, D, chi;
    int op_site[2], op_code[2];
};
// Boundary-MPS workspace (doubles) of one network of this shape.
long long bmps_workspace(int W, int D, int chi);
// Largest boundary bond after a row is applied: max(chi, d) * d, d = D^2.
__host__ __device__ inline int bmps_bond_max(int D, int chi) {
    const int d = D * D;
    return (chi > d ? chi : d) * d;
}
cudaError_t launch_bmps(int dt, const BmpsTask* tasks, int ntasks, cudaStream_t st);   // dt 0: FP64, 1: FP32

// ----------------------------------------------------------- launchers ---
// Each returns cudaSuccess or the launch error.  dt: 0 FP64, 1 FP32.
// variant 0: one outer position per thread (any dtype, K, N); 1 / 2: FP32 with
// K, N in {1, 4, 16}, four outer positions per thread along s (S % 4 == 0) or
// along p (S == 1, P % 4 == 0).  All tasks of one launch share (K, N, variant).
cudaError_t launch_absorb(int dt, bool dot, int K, int N, const AbsorbTask* tasks, int ntasks,
                          long long nblocks, Slot* slots, cudaStream_t st, int variant = 0,
                          const int* tmap = nullptr);
int absorb_variant(int dt, long long P, long long S, int K, int N);
long long absorb_tiles_v(int variant, long long P, long long S, int K, int N);
// Two consecutive steps of one frame row fused (FP32, D = 2: K1 in {4, 16},
// dn, h', u_{c+1} of dimension 4; N2 in {1, 4, 16}): tasks use P = P of the
// first step, S = S of the second, K = K1, N = N2, E = first site matrix,
// E2 = second.
long long absorb2_tiles(long long P, long long S2);
cudaError_t launch_absorb2(bool dot, int K1, int N2, const AbsorbTask* tasks, int ntasks, long long nblocks,
                           Slot* slots, cudaStream_t st, const int* tmap = nullptr);
// variant 0: 64x64 tiles, any dtype; 1: FP32 128x128 double-buffered with
// 16-byte loads; 2: the same with scalar loads (odd extents, e.g. D = 3).
cudaError_t launch_gemm(int dt, bool dot, const GemmTask* tasks, int ntasks, long long nblocks,
                        Slot* slots, cudaStream_t st, int variant = 0);
int gemm_variant(int dt, long long M, long long N, long long K, long long sam, long long sak, long long sbk,
                 long long sbn);
long long gemm_tiles_v(int variant, long long M, long long N, int* tiles_n);
long long gemm_ksplit(int variant, bool dot, long long K);
// Bounded-wait self-check: one thread waits on *flag (never set by the
// library) for at most limit_cycles, then sets *status to 1.
cudaError_t launch_wait_probe(const int* flag, long long limit_cycles, int* status, cudaStream_t st);
// FMA-rate probe: `blocks` blocks of 256 threads, 8 FMA chains x iters each
// (dt 0: FP64 fma; 1: FP32 fma.rn.f32x2, 16 FMAs per round).
cudaError_t launch_fma_probe(int dt, void* out, long long blocks, long long iters, cudaStream_t st);
cudaError_t launch_dot(int dt, const DotTask* tasks, int ntasks, long long nblocks, Slot* slots,
                       cudaStream_t st, const int* tmap = nullptr);
cudaError_t launch_sitemat(int dt, const SiteMatTask* tasks, int ntasks, Slot* slots,
                           cudaStream_t st);
cudaError_t launch_init(Slot* slots, long long nslots, const ConstOne* ones, int nones, int dt,
                        cudaStream_t st);
cudaError_t launch_final(const FinalTask* tasks, int ntasks, const Slot* slots, cudaStream_t st);
// D = 3 interior absorption (K = N = 81) on tensor cores, 512 outer positions per block.
long long tc_absorb_tiles(long long P, long long S);
cudaError_t launch_tc_absorb(int nsplit, bool dot, const AbsorbTask* tasks, int ntasks, long long nblocks,
                             Slot* slots, int* status, cudaStream_t st);
long long tc_split_tiles(long long Rp, long long Kp);
cudaError_t launch_tc_split(const TcSplitTask* tasks, int ntasks, long long nblocks, const Slot* slots,
                            cudaStream_t st);
// status: set to 1 if a bounded wait inside the kernel timed out.
// Output tile 128 x bn, bn = tc_gemm_bn(nsplit, dot, N, Kp): 256 for N > 128
// (the staged bytes per multiply-add halve against 128-wide tiles), except
// short k ranges (Kp <= kTcShortK), which take 128-wide tiles and, when
// stored, a shallow stage ring (launch with short_k) so two CTAs share an SM.
constexpr long long kTcShortK = 1024;
int tc_gemm_bn(int nsplit, bool dot, long long N, long long Kp);
cudaError_t launch_tc_gemm(int nsplit, bool dot, int bn, const TcGemmTask* tasks, int ntasks, long long nblocks,
                           Slot* slots, int* status, cudaStream_t st, bool short_k = false);
// Products fused with a dot (TcGemmTask with ksplit = 1, kchunks = the whole k
// range): one CTA per 128 x bn tile, 512-term slices pipelined through two
// TMEM accumulators (see tc_gemm.cu).  bn from tc_gemm_bn.
cudaError_t launch_tc_gemm_dot(int nsplit, int bn, const TcGemmTask* tasks, int ntasks, long long nblocks,
                               Slot* slots, int* status, cudaStream_t st);
// Rows of every split operand are padded to a multiple of this.
constexpr long long kTcRowPad = 256;
// Reduction (k) width of one staged block of a split operand.
constexpr int kTcChunk = 32;
// Imaginary time evolution (ite.cu): g = {g00, g01, g10, g11} (one-body: the
// 2 x 2 gate; bonds: the diagonal two-body gate g[p_i][p_j]).
cudaError_t launch_ite_one_body(double* A, const long long* site_off, int nsites, const double g[4],
                                cudaStream_t st);
cudaError_t launch_ite_scale(double* A, long long n, const double* log2norm, int nsites, cudaStream_t st);
cudaError_t launch_ite_bonds(double* A, const IteBondTask* tasks, int ntasks, double* ws, const double g[4],
                             int chi_max, double eps, int* kept, unsigned long long* max_disc, cudaStream_t st);
cudaError_t launch_absorb_plain(int dt, const void* in, const void* E, void* out, long long P,
                                int K, int N, long long S, cudaStream_t st);
// <absorb(in, E), adj> into *result (device).  scratch: 16 B counter header
// followed by one double per tile; the caller zeroes the header first.
cudaError_t launch_absorb_dot_plain(int dt, const void* in, const void* E, const void* adj, long long P,
                                    int K, int N, long long S, double* result, void* scratch,
                                    cudaStream_t st);

// Tiles per task, fixed by shape only (bit-identical results alone or batched).
constexpr int kAbsorbThreads = 256;
constexpr int kGemmTile = 64;
constexpr int kDotPerBlock = 4096;
long long absorb_tiles(long long P, long long S, int K, int N);
bool absorb_has_fast_path(int K, int N);
// Variant of the factored D = 3 interior absorption (ket layer, then bra layer).
constexpr int kAbsorbTwoPass = 30;
constexpr int kTwoPassThreads = 128;
long long absorb_2pass_tiles(long long P, long long S);

}  // namespace tn
