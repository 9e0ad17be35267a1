// Ring products on the 5th-generation tensor cores (tcgen05, sm_103a), FP32
// operands split into BF16 planes, FP32 accumulation in tensor memory.
//
// Split (Henry, Tang & Heinecke, "Leveraging the bfloat16 artificial
// intelligence datatype for higher-precision computations", ARITH 2019):
// x = x0 + x1 (+ x2) with x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1);
// a product keeps the terms whose planes sum to at most NSPLIT - 1:
//   NSPLIT = 2: x0 y0 + x0 y1 + x1 y0              (3 tensor-core products)
//   NSPLIT = 3: ... + x0 y2 + x1 y1 + x2 y0         (6 products)
// the smallest terms are accumulated first.
//
// Operand layout ("tiled planes", written by k_tc_split): an R x K operand
// (row r, reduction index k) is padded to multiples of 128 rows and 64 k and
// stored per plane as blocks of 128 rows x 64 k (16 KiB), block (rb, c) at
// ((rb * nchunks) + c) * 16 KiB.  Inside a block the 8x8 core matrices (8 rows
// of 8 consecutive k, 16 bytes per row) are laid out k-fastest: core (ri, ki)
// at (ri * 8 + ki) * 128 bytes.  That is the canonical K-major layout without
// swizzling, so one 16 KiB bulk copy stages a block and the shared-memory
// descriptor uses LBO = 128 B (next core along k) and SBO = 1024 B (next
// 8-row group).
//
// One CTA (128 threads) computes one 128 x 128 output tile: thread 0 of warp 0
// stages k-chunks with cp.async.bulk into a ring of shared-memory stages,
// thread 0 of warp 1 issues the tcgen05.mma and commits each stage back to the
// producer, and all four warps read the accumulator from tensor memory
// (lane = output row) for the epilogue.  Every wait is bounded: on time-out
// the kernel records an error code, drains, frees its tensor memory and exits.
#include <algorithm>
#include <cstdint>

#include <cuda_bf16.h>

#include "ptx.cuh"
#include "pdl.cuh"
#include "tn_kernels.h"

namespace tn {

namespace {

constexpr int kTcM = 128, kTcN = 128, kTcK = kTcChunk;   // tile rows, tile cols, k per chunk
constexpr uint32_t kTcRingBytes = 221184;              // 216 KiB of stage ring (3 x 72 KiB for 3 planes x 256)
constexpr uint32_t kBlockBytes = kTcM * kTcK * 2;     // one 128 x 32 BF16 block (8 KiB)
constexpr uint32_t kTcSBO = (kTcK / 8) * 128;         // next 8-row group inside a block
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, M = 128, N = 128, K = 16, BF16 in, FP32 acc.
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrive on `bar` once every tcgen05 operation issued so far by this thread completes.
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive 32-bit accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: canonical K-major layout, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);             // start address
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;        // LBO: next core matrix along k
    d |= (uint64_t)((kTcSBO >> 4) & 0x3FFF) << 32;      // SBO: next 8-row group
    d |= (uint64_t)1 << 46;                             // descriptor version (tcgen05)
    return d;                                           // base offset 0, no swizzle
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                            ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ int slot_shift_tc(const Slot* s) {
    const double m = __longlong_as_double((long long)s->maxbits);
    if (!(m > 0.0)) return 0;
    int e;
    frexp(m, &e);
    return e;
}

__device__ __forceinline__ float pow2f(int e) {
    e = e < -125 ? -125 : (e > 125 ? 125 : e);
    return __int_as_float((127 + e) << 23);
}

template <typename Task>
__device__ __forceinline__ int find_task_tc(const Task* __restrict__ tasks, int ntasks, long long tile) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct CSumF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        c += (fabsf(s) >= fabsf(x)) ? (s - t) + x : (x - t) + s;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s + c; }
};

__device__ __forceinline__ double block_reduce(double v, double* red, bool is_max) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, w) : v + w;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = is_max ? 0.0 : 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = is_max ? fmax(r, red[k]) : r + red[k];
    return r;
}

}  // namespace

// ----------------------------------------------------------------- split --

// One thread per (row, 8-wide k group) of the padded operand.
__global__ void __launch_bounds__(256)
k_tc_split(const TcSplitTask* __restrict__ tasks, int ntasks, const Slot* __restrict__ slots) {
    pdl_enter();
    const long long tile = blockIdx.x;
    const TcSplitTask& t = tasks[find_task_tc(tasks, ntasks, tile)];
    const long long idx = (tile - t.tile0) * 256 + threadIdx.x;
    const long long nko = t.Kp / 8;
    if (idx >= t.Rp * nko) return;
    const long long r = idx % t.Rp, ko = idx / t.Rp;   // consecutive threads: consecutive rows
    const float sc = pow2f(-slot_shift_tc(&slots[t.slot_src]));
    const float* src = static_cast<const float*>(t.src);
    float x[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const long long k = ko * 8 + kk;
        x[kk] = (r < t.R && k < t.Kd) ? src[r * t.sr + k * t.sk] * sc : 0.0f;
    }
    constexpr int kOct = kTcK / 8;                    // 8-wide k groups per chunk
    const long long nchunks = t.Kp / kTcK;
    const long long rb = r / kTcM, rr = r % kTcM, c = ko / kOct, ki = ko % kOct;
    const long long off = (rb * nchunks + c) * (long long)kBlockBytes + (((rr / 8) * kOct + ki) * 8 + (rr % 8)) * 16;
    __align__(16) __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[kk]);
        const float r1 = x[kk] - __bfloat162float(h0);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(h1);
        p0[kk] = h0;
        p1[kk] = h1;
        p2[kk] = __float2bfloat16_rn(r2);
    }
    char* dst = static_cast<char*>(t.dst);
    *reinterpret_cast<uint4*>(dst + off) = *reinterpret_cast<const uint4*>(p0);
    *reinterpret_cast<uint4*>(dst + t.plane_bytes + off) = *reinterpret_cast<const uint4*>(p1);
    if (t.nsplit == 3) *reinterpret_cast<uint4*>(dst + 2 * t.plane_bytes + off) = *reinterpret_cast<const uint4*>(p2);
}

// ------------------------------------------------------------------ mma ---

// STAGES: ring depth (0: as many 192 KB allow, up to 6; short k ranges use a
// shallow ring so two CTAs share an SM and overlap each other's epilogues).
template <int NSPLIT, bool DOT, int BN, int STAGES_>
__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const TcGemmTask* __restrict__ tasks, int ntasks, Slot* __restrict__ slots, int* __restrict__ status) {
    pdl_enter();
    constexpr int NB = BN / kTcM;                                   // 128-row B blocks per tile
    constexpr uint32_t kStageBytes = NSPLIT * (1 + NB) * kBlockBytes;   // A planes then B planes
    constexpr int STAGES =
        STAGES_ > 0 ? STAGES_ : ((kTcRingBytes / kStageBytes) >= 6 ? 6 : (int)(kTcRingBytes / kStageBytes));
    constexpr int NPROD = NSPLIT == 2 ? 3 : 6;
    // products (plane of A, plane of B), smallest terms first
    constexpr int PA[6] = {NSPLIT == 2 ? 1 : 2, NSPLIT == 2 ? 0 : 1, NSPLIT == 2 ? 0 : 0, 1, 0, 0};
    constexpr int PB[6] = {NSPLIT == 2 ? 0 : 0, NSPLIT == 2 ? 1 : 1, NSPLIT == 2 ? 0 : 2, 0, 1, 0};
    constexpr uint32_t kIdescN = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                 ((uint32_t)(kTcM >> 4) << 24);
    constexpr int kGroup = 8;                                       // tile rows sharing A in L2
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;
    __shared__ double red[32];

    const long long tile = blockIdx.x;
    const TcGemmTask& t = tasks[find_task_tc(tasks, ntasks, tile)];
    const long long local = tile - t.tile0;
    const long long mn = local / t.ksplit, ks = local % t.ksplit;
    // grouped rasterisation: kGroup tile rows, columns outer, rows inner
    const long long per_group = (long long)kGroup * t.tiles_n;
    const long long g = mn / per_group, gi = mn % per_group;
    const long long grows = min((long long)kGroup, t.tiles_m - g * kGroup);
    const long long tm = g * kGroup + gi % grows, tn_ = gi / grows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long nchunks_all = t.Kp / kTcK;       // chunks of the whole k range (layout)
    const long long cbeg = ks * t.kchunks;
    const long long nchunks = min(nchunks_all, cbeg + t.kchunks) - cbeg;
    // 1024-byte aligned start of the stage ring
    unsigned char* ring = smem + ((1024 - (smem_u32(smem) & 1023)) & 1023);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        mbar_init(&done_bar, 1);
        fail_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_sh, BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    const char* Ab = static_cast<const char*>(t.A) + (tm * nchunks_all + cbeg) * (long long)kBlockBytes;
    const char* Bb = static_cast<const char*>(t.B) + (tn_ * NB * nchunks_all + cbeg) * (long long)kBlockBytes;
    int my_fail = 0;
    int armed[STAGES];
#pragma unroll
    for (int s = 0; s < STAGES; ++s) armed[s] = 0;
    if (warp == 0 && lane == 0) {
        // producer: stage k-chunk c into ring slot c % STAGES
        for (long long c = 0; c < nchunks && !my_fail; ++c) {
            const int s = (int)(c % STAGES);
            if (c >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)((c / STAGES - 1) & 1))) { my_fail = 1; break; }
            unsigned char* st = ring + s * kStageBytes;
            armed[s] += 1;
            mbar_expect_tx(&full_bar[s], kStageBytes);
            for (int p = 0; p < NSPLIT; ++p) {
                bulk_g2s(st + p * kBlockBytes, Ab + p * t.a_plane_bytes + c * kBlockBytes, kBlockBytes, &full_bar[s]);
                // the NB row blocks of B sit back to back, so one descriptor spans them
                for (int h = 0; h < NB; ++h)
                    bulk_g2s(st + (NSPLIT + p * NB + h) * kBlockBytes,
                             Bb + p * t.b_plane_bytes + (h * nchunks_all + c) * kBlockBytes, kBlockBytes,
                             &full_bar[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        for (long long c = 0; c < nchunks; ++c) {
            const int s = (int)(c % STAGES);
            if (!mbar_wait(&full_bar[s], (uint32_t)((c / STAGES) & 1))) { my_fail = 1; break; }
            tc_fence_after();
            const uint32_t st = smem_u32(ring + s * kStageBytes);
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk) {
#pragma unroll
                for (int q = 0; q < NPROD; ++q) {
                    const uint64_t da = smem_desc(st + PA[q] * kBlockBytes + kk * 256);
                    const uint64_t db = smem_desc(st + (NSPLIT + PB[q] * NB) * kBlockBytes + kk * 256);
                    tc_mma(tmem, da, db, kIdescN, (c > 0 || kk > 0 || q > 0) ? 1u : 0u);
                }
            }
            tc_commit(&empty_bar[s]);
        }
        tc_commit(&done_bar);
    }
    if (my_fail) atomicExch(&fail_sh, 1);
    // epilogue: wait for the last MMA (bounded), then read the accumulator
    bool ok = mbar_wait(&done_bar, 0u);
    __syncthreads();
    if (!ok || fail_sh) {
        if (threadIdx.x == 0) atomicExch(status, 1);
        // never leave with our own bulk copies in flight: wait (bounded) for the
        // last phase the producer armed on every stage
        if (warp == 0 && lane == 0)
            for (int s = 0; s < STAGES; ++s)
                if (armed[s] > 0) (void)mbar_wait(&full_bar[s], (uint32_t)((armed[s] - 1) & 1));
    }
    __syncthreads();
    tc_fence_after();
    const long long row = tm * kTcM + warp * 32 + lane;
    const long long n0 = tn_ * BN;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    const int eA = slot_shift_tc(&slots[t.slot_A]), eB = slot_shift_tc(&slots[t.slot_B]);
    double mx = 0.0, dsum = 0.0;
    const bool good = ok && !fail_sh;
    float sD = 1.0f;
    int eD = 0;
    if (DOT) { eD = slot_shift_tc(&slots[t.slot_D]); sD = pow2f(-eD); }
    for (int cb = 0; cb < BN; cb += 16) {
        float v[16];
        tmem_ld16(lane_addr + (uint32_t)cb, v);
        if (!good || row >= t.M) continue;
        if (!DOT) {
            float* C = static_cast<float*>(t.C) + row * t.N;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const long long n = n0 + cb + i;
                if (n < t.N) { C[n] = v[i]; mx = fmax(mx, (double)fabsf(v[i])); }
            }
        } else {
            const float* Dm = static_cast<const float*>(t.Dm) + row * t.N;
            float s = 0.0f, comp = 0.0f;    // compensated (Neumaier) sum of 16 products
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const long long n = n0 + cb + i;
                if (n < t.N) {
                    const float x = v[i] * (Dm[n] * sD), tt = s + x;
                    comp += (fabsf(s) >= fabsf(x)) ? (s - tt) + x : (x - tt) + s;
                    s = tt;
                }
            }
            dsum += (double)s + (double)comp;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, BN);
    if (!DOT) {
        const double m = block_reduce(mx, red, true);
        if (threadIdx.x == 0) {
            atomicMax(&slots[t.slot_C].maxbits, (unsigned long long)__double_as_longlong(m));
            if (local == 0) slots[t.slot_C].X = slots[t.slot_A].X + eA + slots[t.slot_B].X + eB;
        }
    } else {
        const double part = block_reduce(dsum, red, false);
        __shared__ int is_last;
        if (threadIdx.x == 0) {
            t.partial[local] = part;
            __threadfence();
            const unsigned prev = atomicAdd(&slots[t.slot_C].count, 1u);
            is_last = (prev == (unsigned)(t.ntiles - 1));
        }
        __syncthreads();
        if (is_last) {
            __threadfence();
            double acc = 0.0;
            for (int k = threadIdx.x; k < t.ntiles; k += blockDim.x) acc += __ldcg(t.partial + k);
            acc = block_reduce(acc, red, false);
            if (threadIdx.x == 0) {
                slots[t.slot_C].mant = acc;
                slots[t.slot_C].X = slots[t.slot_A].X + eA + slots[t.slot_B].X + eB + slots[t.slot_D].X + eD;
            }
        }
    }
}

// ---- products fused with a dot: whole k range per CTA, slices pipelined ----
//
// <A B^T, Dm> over one 128 x BN output tile: the k range is cut into slices
// of kGemmKSlice (512) terms; the tensor cores accumulate slice s into one of
// two TMEM accumulators while four epilogue warps take the other: each reads
// its rows of slice s - 1's product, forms the compensated FP32 dot with its
// rows of Dm and adds it to an FP64 sum -- the same numerics as one CTA per
// slice, without refilling the pipeline for every 512 terms.  Warp 0 stages
// k-chunks (thread 0, cp.async.bulk), warp 1 issues the MMAs (thread 0) and
// owns the tensor memory, warps 2.. are the epilogue: BN / 32 warps, warp w
// reads TMEM lanes 32 (w mod 4) .. for the 128 columns (w - 2) / 4 and holds
// that part of its row of the Dm tile in registers for every slice.  One FP64
// partial per tile; the last tile to finish
// sums them in index order.  Every wait is bounded; on a time-out the kernel
// records the error, waits (bounded) for its copies and MMAs, frees its
// tensor memory and exits.
constexpr int kDotSlice = (int)(kGemmKSlice / kTcK);   // chunks per slice
__host__ __device__ constexpr int dot_threads(int bn) { return 64 + 32 * (bn / 32); }

template <int NSPLIT, int BN, int STAGES>
__global__ void __launch_bounds__(dot_threads(BN), 1)
k_tc_gemm_dot(const TcGemmTask* __restrict__ tasks, int ntasks, Slot* __restrict__ slots, int* __restrict__ status) {
    pdl_enter();
    constexpr int NB = BN / kTcM;
    constexpr uint32_t kStageBytes = NSPLIT * (1 + NB) * kBlockBytes;
    constexpr int NPROD = NSPLIT == 2 ? 3 : 6;
    constexpr int PA[6] = {NSPLIT == 2 ? 1 : 2, NSPLIT == 2 ? 0 : 1, NSPLIT == 2 ? 0 : 0, 1, 0, 0};
    constexpr int PB[6] = {NSPLIT == 2 ? 0 : 0, NSPLIT == 2 ? 1 : 1, NSPLIT == 2 ? 0 : 2, 0, 1, 0};
    constexpr uint32_t kIdescN = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                                 ((uint32_t)(kTcM >> 4) << 24);
    constexpr int kGroup = 8;
    constexpr int kEpiWarps = BN / 32;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_full[2], acc_empty[2], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;
    __shared__ double red[dot_threads(BN) / 32];
    __shared__ int is_last;

    const long long tile = blockIdx.x;
    const TcGemmTask& t = tasks[find_task_tc(tasks, ntasks, tile)];
    const long long local = tile - t.tile0;
    const long long per_group = (long long)kGroup * t.tiles_n;
    const long long g = local / per_group, gi = local % per_group;
    const long long grows = min((long long)kGroup, t.tiles_m - g * kGroup);
    const long long tm = g * kGroup + gi % grows, tn_ = gi / grows;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long nchunks = t.Kp / kTcK;
    const int nslices = (int)((nchunks + kDotSlice - 1) / kDotSlice);
    unsigned char* ring = smem + ((1024 - (smem_u32(smem) & 1023)) & 1023);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], kEpiWarps); }
        mbar_init(&done_bar, 1);
        fail_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        tmem_alloc(&tmem_base_sh, 2 * BN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    const char* Ab = static_cast<const char*>(t.A) + tm * nchunks * (long long)kBlockBytes;
    const char* Bb = static_cast<const char*>(t.B) + tn_ * NB * nchunks * (long long)kBlockBytes;
    int armed[STAGES];
#pragma unroll
    for (int s = 0; s < STAGES; ++s) armed[s] = 0;
    double dsum = 0.0;
    if (warp == 0) {
        if (lane == 0) {
            for (long long c = 0; c < nchunks; ++c) {
                const int s = (int)(c % STAGES);
                if (c >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)((c / STAGES - 1) & 1))) {
                    atomicExch(&fail_sh, 1);
                    break;
                }
                if (*(volatile int*)&fail_sh) break;
                unsigned char* st = ring + s * kStageBytes;
                armed[s] += 1;
                mbar_expect_tx(&full_bar[s], kStageBytes);
                for (int p = 0; p < NSPLIT; ++p) {
                    bulk_g2s(st + p * kBlockBytes, Ab + p * t.a_plane_bytes + c * kBlockBytes, kBlockBytes,
                             &full_bar[s]);
                    for (int h = 0; h < NB; ++h)
                        bulk_g2s(st + (NSPLIT + p * NB + h) * kBlockBytes,
                                 Bb + p * t.b_plane_bytes + (h * nchunks + c) * kBlockBytes, kBlockBytes,
                                 &full_bar[s]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (long long c = 0; c < nchunks; ++c) {
                const int sl = (int)(c / kDotSlice), buf = sl & 1;
                const bool first = (c % kDotSlice) == 0;
                if (first && sl >= 2 && !mbar_wait(&acc_empty[buf], (uint32_t)((sl / 2 - 1) & 1))) {
                    atomicExch(&fail_sh, 1);
                    break;
                }
                const int s = (int)(c % STAGES);
                if (!mbar_wait(&full_bar[s], (uint32_t)((c / STAGES) & 1))) { atomicExch(&fail_sh, 1); break; }
                if (*(volatile int*)&fail_sh) break;
                tc_fence_after();
                const uint32_t stg = smem_u32(ring + s * kStageBytes);
                const uint32_t acc = tmem + (uint32_t)(buf * BN);
#pragma unroll
                for (int kk = 0; kk < kTcK / 16; ++kk) {
#pragma unroll
                    for (int q = 0; q < NPROD; ++q) {
                        const uint64_t da = smem_desc(stg + PA[q] * kBlockBytes + kk * 256);
                        const uint64_t db = smem_desc(stg + (NSPLIT + PB[q] * NB) * kBlockBytes + kk * 256);
                        tc_mma(acc, da, db, kIdescN, (!first || kk > 0 || q > 0) ? 1u : 0u);
                    }
                }
                tc_commit(&empty_bar[s]);
                if ((c % kDotSlice) == kDotSlice - 1 || c == nchunks - 1) tc_commit(&acc_full[buf]);
            }
            tc_commit(&done_bar);
        }
    } else {
        // epilogue: warps 2.., TMEM lane quadrant warp % 4, 128 columns (warp - 2) / 4
        const int quad = warp & 3, half = (warp - 2) >> 2;
        const long long row = tm * kTcM + quad * 32 + lane;
        const long long n0 = tn_ * BN + half * 128;
        const int eD = slot_shift_tc(&slots[t.slot_D]);
        const float sD = pow2f(-eD);
        // this thread's row of the Dm tile, rescaled, held in registers for every slice
        // (zero beyond the matrix, so padded rows and columns add nothing)
        float dm[128];
        {
            const float* Dm = static_cast<const float*>(t.Dm) + row * t.N;
#pragma unroll
            for (int i = 0; i < 128; ++i) {
                const long long n = n0 + i;
                dm[i] = (row < t.M && n < t.N) ? __ldg(Dm + n) * sD : 0.0f;
            }
        }
        for (int sl = 0; sl < nslices; ++sl) {
            const int buf = sl & 1;
            if (!mbar_wait(&acc_full[buf], (uint32_t)((sl / 2) & 1))) { atomicExch(&fail_sh, 1); break; }
            tc_fence_after();
            const uint32_t lane_addr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BN + half * 128);
            float s = 0.0f, comp = 0.0f;     // compensated (Neumaier) sum of this slice's products
#pragma unroll
            for (int cb = 0; cb < 128; cb += 16) {
                float v[16];
                tmem_ld16(lane_addr + (uint32_t)cb, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const float x = v[i] * dm[cb + i], tt = s + x;
                    comp += (fabsf(s) >= fabsf(x)) ? (s - tt) + x : (x - tt) + s;
                    s = tt;
                }
            }
            dsum += (double)s + (double)comp;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[buf]);
        }
    }
    // every MMA issued has completed (bounded), and no copy is left in flight
    const bool ok = mbar_wait(&done_bar, 0u);
    if (!ok) atomicExch(&fail_sh, 1);
    __syncthreads();
    const bool failed = *(volatile int*)&fail_sh != 0;
    if (failed) {
        if (threadIdx.x == 0) atomicExch(status, 1);
        if (warp == 0 && lane == 0)
            for (int s = 0; s < STAGES; ++s)
                if (armed[s] > 0) (void)mbar_wait(&full_bar[s], (uint32_t)((armed[s] - 1) & 1));
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem, 2 * BN);
    if (failed) return;
    const int eA = slot_shift_tc(&slots[t.slot_A]), eB = slot_shift_tc(&slots[t.slot_B]);
    const double part = block_reduce(dsum, red, false);
    if (threadIdx.x == 0) {
        t.partial[local] = part;
        __threadfence();
        const unsigned prev = atomicAdd(&slots[t.slot_C].count, 1u);
        is_last = (prev == (unsigned)(t.ntiles - 1));
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        double accp = 0.0;
        for (int k = threadIdx.x; k < t.ntiles; k += blockDim.x) accp += __ldcg(t.partial + k);
        accp = block_reduce(accp, red, false);
        if (threadIdx.x == 0) {
            const int eD = slot_shift_tc(&slots[t.slot_D]);
            slots[t.slot_C].mant = accp;
            slots[t.slot_C].X = slots[t.slot_A].X + eA + slots[t.slot_B].X + eB + slots[t.slot_D].X + eD;
        }
    }
}

// ------------------------------------------------------- D=3 absorption --
//
// Out[p][n][s] = sum_k In[p][k][s] E[k][n] for K = N = 81 (interior double-layer
// steps of D = 3) on tensor cores.  Each CTA (128 threads) takes kAbsSub
// consecutive groups of 128 outer positions o = p*S + s.  Per group, thread t
// loads the 81 inputs of position o0 + t (rescaled by the input slot), splits
// them into BF16 planes and writes them as row t of the A operand (K-major,
// k padded to 96); the site matrix, transposed into B'[n][k], is split once per
// CTA.  One thread issues 6 k-steps x NPROD products (M = 128, N = 96), the
// accumulator row of each lane is its outer position, so the FP32 stores of
// Out (or the fused dot with the adjoint) are coalesced along s.
constexpr int kAbsK = 81, kAbsKp = 96, kAbsSub = 4;
constexpr uint32_t kAbsAPlane = 128 * kAbsKp * 2;   // 24 KiB
constexpr uint32_t kAbsBPlane = kAbsKp * kAbsKp * 2;  // 18 KiB
constexpr uint32_t kAbsSBO = (kAbsKp / 8) * 128;      // next 8-row group: 12 core matrices
constexpr uint32_t kAbsIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kAbsKp >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint64_t smem_desc_sbo(uint32_t saddr, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Split 8 FP32 values and store them as one 16-byte row segment per plane.
template <int NSPLIT>
__device__ __forceinline__ void split_store8(const float* x, unsigned char* base, uint32_t plane_bytes, uint32_t off) {
    __align__(16) __nv_bfloat16 q0[8], q1[8], q2[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[i]);
        const float r1 = x[i] - __bfloat162float(h0);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
        q0[i] = h0;
        q1[i] = h1;
        if (NSPLIT == 3) q2[i] = __float2bfloat16_rn(r1 - __bfloat162float(h1));
    }
    *reinterpret_cast<uint4*>(base + off) = *reinterpret_cast<const uint4*>(q0);
    *reinterpret_cast<uint4*>(base + plane_bytes + off) = *reinterpret_cast<const uint4*>(q1);
    if (NSPLIT == 3) *reinterpret_cast<uint4*>(base + 2 * plane_bytes + off) = *reinterpret_cast<const uint4*>(q2);
}

template <int NSPLIT, int MODE>
__global__ void __launch_bounds__(128, 1)
k_tc_absorb(const AbsorbTask* __restrict__ tasks, int ntasks, Slot* __restrict__ slots, int* __restrict__ status) {
    pdl_enter();
    constexpr int NPROD = NSPLIT == 2 ? 3 : 6;
    constexpr int PA[6] = {NSPLIT == 2 ? 1 : 2, NSPLIT == 2 ? 0 : 1, NSPLIT == 2 ? 0 : 0, 1, 0, 0};
    constexpr int PB[6] = {NSPLIT == 2 ? 0 : 0, NSPLIT == 2 ? 1 : 1, NSPLIT == 2 ? 0 : 2, 0, 1, 0};
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mma_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ double red[32];
    unsigned char* ring = smem + ((1024 - (smem_u32(smem) & 1023)) & 1023);
    unsigned char* Bs = ring;                                  // NSPLIT planes of B'
    unsigned char* As = ring + NSPLIT * kAbsBPlane;            // NSPLIT planes of A

    const long long tile = blockIdx.x;
    const AbsorbTask& t = tasks[find_task_tc(tasks, ntasks, tile)];
    const long long local = tile - t.tile0;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long S = t.S, nouter = t.P * S;

    if (tid == 0) {
        mbar_init(&mma_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_sh, 128);
        tmem_relinquish();
    }
    // B'[n][k] = E_task[k][n], zero outside 81 x 81
    const float* E = static_cast<const float*>(t.E);
    if (tid < kAbsKp) {
#pragma unroll 1
        for (int k8 = 0; k8 < kAbsKp / 8; ++k8) {
            float x[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int k = 8 * k8 + i, n = tid;
                x[i] = (k < kAbsK && n < kAbsK) ? (t.transE ? E[n * kAbsK + k] : E[k * kAbsK + n]) : 0.0f;
            }
            split_store8<NSPLIT>(x, Bs, kAbsBPlane, (uint32_t)(((tid >> 3) * (kAbsKp / 8) + k8) * 128 + (tid & 7) * 16));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int e_in = slot_shift_tc(&slots[t.slot_in]);
    const float sc_in = pow2f(-e_in);
    int e_adj = 0;
    float sc_adj = 1.0f;
    if (MODE == 2) { e_adj = slot_shift_tc(&slots[t.slot_adj]); sc_adj = pow2f(-e_adj); }
    const float* in = static_cast<const float*>(t.in);
    float lmax = 0.0f;
    double ldot = 0.0;
    bool ok = true;
    int last_fail = -1;
    for (int sub = 0; sub < kAbsSub; ++sub) {
        const long long o = (local * kAbsSub + sub) * 128 + tid;
        const bool valid = o < nouter;
        const long long p = valid ? o / S : 0, s = valid ? o - p * S : 0;
        // A row tid: the 81 inputs of this outer position (k padded to 96)
        float x[kAbsKp];
#pragma unroll
        for (int k = 0; k < kAbsKp; ++k) x[k] = (valid && k < kAbsK) ? in[(p * kAbsK + k) * S + s] * sc_in : 0.0f;
#pragma unroll
        for (int k8 = 0; k8 < kAbsKp / 8; ++k8)
            split_store8<NSPLIT>(x + 8 * k8, As, kAbsAPlane,
                                 (uint32_t)(((tid >> 3) * (kAbsKp / 8) + k8) * 128 + (tid & 7) * 16));
        // make the generic-proxy stores visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
            for (int ks = 0; ks < kAbsKp / 16; ++ks)
#pragma unroll
                for (int q = 0; q < NPROD; ++q)
                    tc_mma(tmem, smem_desc_sbo(a0 + PA[q] * kAbsAPlane + ks * 256, kAbsSBO),
                           smem_desc_sbo(b0 + PB[q] * kAbsBPlane + ks * 256, kAbsSBO), kAbsIdesc,
                           (ks > 0 || q > 0) ? 1u : 0u);
            tc_commit(&mma_bar);
        }
        // bounded wait; the verdict is made block-uniform so all warps stop together
        ok = __syncthreads_and(mbar_wait(&mma_bar, (uint32_t)(sub & 1)) ? 1 : 0) != 0;
        if (!ok) {
            last_fail = sub;
            break;
        }
        tc_fence_after();
        // accumulator lane = this warp's rows; 6 x 16 columns
        const long long orow = (local * kAbsSub + sub) * 128 + warp * 32 + lane;
        const bool vrow = orow < nouter;
        const long long pr = vrow ? orow / S : 0, sr = vrow ? orow - pr * S : 0;
        CSumF acc;
#pragma unroll
        for (int cb = 0; cb < kAbsKp; cb += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
            if (!vrow) continue;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = cb + i;
                if (n >= kAbsK) continue;
                const long long idx = (pr * kAbsK + n) * S + sr;
                if (MODE == 1) {
                    static_cast<float*>(t.out)[idx] = v[i];
                    lmax = fmaxf(lmax, fabsf(v[i]));
                } else {
                    acc.add(v[i] * (static_cast<const float*>(t.adj)[idx] * sc_adj));
                }
            }
        }
        if (MODE == 2) ldot += (double)acc.value();
        // every thread has read its accumulator lanes before the next group overwrites A or D
        tc_fence_before();
        __syncthreads();
    }
    if (!ok) {
        // the products of the failed group may still run: wait for them once
        // more (bounded) before the tensor memory is returned
        if (tid == 0) {
            atomicExch(status, 1);
            (void)mbar_wait(&mma_bar, (uint32_t)(last_fail & 1));
        }
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 128);
    if (MODE == 1) {
        const double m = block_reduce((double)lmax, red, true);
        if (tid == 0) {
            atomicMax(&slots[t.slot_out].maxbits, (unsigned long long)__double_as_longlong(m));
            if (local == 0) slots[t.slot_out].X = slots[t.slot_in].X + e_in + slots[t.slot_E].X;
        }
    } else {
        const double part = block_reduce(ldot, red, false);
        __shared__ int is_last;
        if (tid == 0) {
            t.partial[local] = part;
            __threadfence();
            const unsigned prev = atomicAdd(&slots[t.slot_out].count, 1u);
            is_last = (prev == (unsigned)(t.ntiles - 1));
        }
        __syncthreads();
        if (is_last) {
            __threadfence();
            double a = 0.0;
            for (int k = tid; k < t.ntiles; k += blockDim.x) a += __ldcg(t.partial + k);
            a = block_reduce(a, red, false);
            if (tid == 0) {
                slots[t.slot_out].mant = a;
                slots[t.slot_out].X =
                    slots[t.slot_in].X + e_in + slots[t.slot_E].X + slots[t.slot_adj].X + e_adj;
            }
        }
    }
}

long long tc_absorb_tiles(long long P, long long S) { return (P * S + 128 * kAbsSub - 1) / (128 * kAbsSub); }

cudaError_t launch_tc_absorb(int nsplit, bool dot, const AbsorbTask* tasks, int ntasks, long long nblocks,
                             Slot* slots, int* status, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    if (nsplit != 2 && nsplit != 3) return cudaErrorInvalidValue;
    const size_t smem = (size_t)nsplit * (kAbsAPlane + kAbsBPlane) + 1024;
#define TN_TCA_LAUNCH(NS, MD)                                                                  \
    {                                                                                          \
        auto fn = k_tc_absorb<NS, MD>;                                                         \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                        \
        TN_LAUNCH(fn, dim3((unsigned)nblocks), dim3(128), smem, st, tasks, ntasks, slots, status);                \
        return cudaGetLastError();                                                             \
    }
    if (nsplit == 2) { if (dot) TN_TCA_LAUNCH(2, 2) else TN_TCA_LAUNCH(2, 1) }
    if (dot) TN_TCA_LAUNCH(3, 2) else TN_TCA_LAUNCH(3, 1)
#undef TN_TCA_LAUNCH
}

// ------------------------------------------------------------- launchers --

long long tc_split_tiles(long long Rp, long long Kp) { return (Rp * (Kp / 8) + 255) / 256; }

// One kernel of this translation unit, for loading its module up front (preload.cpp).
const void* tc_module_anchor() { return reinterpret_cast<const void*>(&k_tc_split); }

cudaError_t launch_tc_split(const TcSplitTask* tasks, int ntasks, long long nblocks, const Slot* slots,
                            cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    TN_LAUNCH(k_tc_split, dim3((unsigned)nblocks), dim3(256), 0, st, tasks, ntasks, slots);
    return cudaGetLastError();
}

cudaError_t launch_tc_gemm_dot(int nsplit, int bn, const TcGemmTask* tasks, int ntasks, long long nblocks,
                               Slot* slots, int* status, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    const int nb = bn / kTcM;
    const uint32_t stage = (uint32_t)nsplit * (1 + nb) * kBlockBytes;
    // as many stages as 216 KiB hold, at most 4 (3 for 3 planes x 256)
    const int stages = (int)std::min<uint32_t>(4, kTcRingBytes / stage);
    const size_t smem = (size_t)stages * stage + 1024;
#define TN_TCD_LAUNCH(NS, B)                                                                   \
    {                                                                                          \
        auto fn = k_tc_gemm_dot<NS, B, (NS) * (1 + (B) / 128) * 8192 * 4 <= (int)kTcRingBytes ? 4 : 3>; \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                        \
        TN_LAUNCH(fn, dim3((unsigned)nblocks), dim3(dot_threads(B)), smem, st, tasks, ntasks, slots, status); \
        return cudaGetLastError();                                                             \
    }
    if (nsplit == 2 && bn == 256) TN_TCD_LAUNCH(2, 256)
    if (nsplit == 3 && bn == 256) TN_TCD_LAUNCH(3, 256)
    if (nsplit == 2 && bn == 128) TN_TCD_LAUNCH(2, 128)
    if (nsplit == 3 && bn == 128) TN_TCD_LAUNCH(3, 128)
#undef TN_TCD_LAUNCH
    return cudaErrorInvalidValue;
}

int tc_gemm_bn(int nsplit, bool dot, long long N, long long Kp) {
    (void)nsplit; (void)dot;
    if (Kp <= kTcShortK) return 128;
    return N > 128 ? 256 : 128;
}

cudaError_t launch_tc_gemm(int nsplit, bool dot, int bn, const TcGemmTask* tasks, int ntasks, long long nblocks,
                           Slot* slots, int* status, cudaStream_t st, bool short_k) {
    if (nblocks <= 0) return cudaSuccess;
    const int nb = bn / kTcM;
    const uint32_t stage = (uint32_t)nsplit * (1 + nb) * kBlockBytes;
    const int stages = short_k ? (nsplit == 2 ? 3 : 2) : ((kTcRingBytes / stage) >= 6 ? 6 : (int)(kTcRingBytes / stage));
    const size_t smem = (size_t)stages * stage + 1024;
    if (short_k) {
        // 128-wide tiles, 2 (3 planes) or 3 (2 planes) stages: ~97 KB, two CTAs per SM
#define TN_TCS_LAUNCH(NS, DT, SG)                                                              \
        {                                                                                      \
            auto fn = k_tc_gemm<NS, DT, 128, SG>;                                              \
            cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            if (e != cudaSuccess) return e;                                                    \
            TN_LAUNCH(fn, dim3((unsigned)nblocks), dim3(128), smem, st, tasks, ntasks, slots, status);            \
            return cudaGetLastError();                                                         \
        }
        if (bn != 128) return cudaErrorInvalidValue;
        if (dot) return cudaErrorInvalidValue;
        if (nsplit == 2) TN_TCS_LAUNCH(2, false, 3)
        TN_TCS_LAUNCH(3, false, 2)
#undef TN_TCS_LAUNCH
    }
#define TN_TC_LAUNCH(NS, DT, B)                                                                \
    {                                                                                          \
        auto fn = k_tc_gemm<NS, DT, B, 0>;                                                     \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                        \
        TN_LAUNCH(fn, dim3((unsigned)nblocks), dim3(128), smem, st, tasks, ntasks, slots, status);                \
        return cudaGetLastError();                                                             \
    }
    // products fused with a dot go to launch_tc_gemm_dot; this kernel stores
    if (dot) return cudaErrorInvalidValue;
    if (nsplit == 2 && bn == 256) TN_TC_LAUNCH(2, false, 256)
    if (nsplit == 3 && bn == 256) TN_TC_LAUNCH(3, false, 256)
    if (nsplit == 2) TN_TC_LAUNCH(2, false, 128)
    TN_TC_LAUNCH(3, false, 128)
#undef TN_TC_LAUNCH
}

}  // namespace tn
