// Block-wide one-sided Jacobi SVD (Hestenes 1958; Demmel & Veselic 1992) on a
// matrix in global memory, FP64 or FP32.  The n columns of A (column-major, leading
// dimension lda, m rows) are rotated pairwise until mutually orthogonal; the
// same rotations applied to V (n x n, column-major, leading dimension ldv,
// reset to the identity here) give A_in = A_out V^T with A_out = U Sigma, so
// sigma_c = |column c of A_out|.  Pairs follow the round-robin (circle)
// schedule: n2 - 1 rounds of n2 / 2 disjoint pairs per sweep (n2 = n rounded
// up to even, the extra column treated as zero), one warp per pair, in a fixed
// order, so a result is reproducible.  A sweep in which no pair needed a
// rotation (|a.b| <= 1e-15 |a| |b| for every pair) ends the iteration.
// Every thread of the block must call it; it synchronises the block.
#pragma once

namespace tn {

constexpr int kJacobiMaxSweeps = 60;

template <typename T>
__device__ __forceinline__ T jacobi_warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// `flag` is one int of shared memory owned by the caller.  T is double or
// float; a pair counts as orthogonal when |a.b| <= tol |a| |b|, tol = 1e-15
// (double) or 1e-6 (float, a few units of its rounding).  A column whose norm
// is at most tol |A|_F is numerically zero (the matrices here are often rank-
// deficient, e.g. a two-site product through a bond of dimension chi): its
// pairs are not rotated, so rounding noise in such columns cannot keep the
// sweeps from converging.
template <typename T>
__device__ inline void block_jacobi(T* A, int m, int n, long long lda, T* V, long long ldv, int* flag) {
    const T tol = sizeof(T) == 8 ? T(1e-15) : T(1e-6);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int n2 = n + (n & 1);
    __shared__ T fro_part[32];
    T f2 = 0;
    for (long long idx = threadIdx.x; idx < (long long)n * m; idx += blockDim.x) {
        const int c = (int)(idx / m), r = (int)(idx - (long long)c * m);
        const T x = A[c * lda + r];
        f2 += x * x;
    }
    f2 = jacobi_warp_sum(f2);
    if (lane == 0) fro_part[warp] = f2;
    for (long long idx = threadIdx.x; idx < (long long)n * n; idx += blockDim.x) {
        const int c = (int)(idx / n), r = (int)(idx - (long long)c * n);
        V[c * ldv + r] = r == c ? T(1) : T(0);
    }
    __syncthreads();
    T fro2 = 0;
    for (int w = 0; w < nwarps; ++w) fro2 += fro_part[w];
    const T negligible = tol * tol * fro2;
    __syncthreads();
    for (int sweep = 0; sweep < kJacobiMaxSweeps && n > 1; ++sweep) {
        if (threadIdx.x == 0) *flag = 1;
        __syncthreads();
        for (int round = 0; round < n2 - 1; ++round) {
            for (int k = warp; k < n2 / 2; k += nwarps) {
                int a, b;
                if (k == 0) { a = round; b = n2 - 1; }
                else { a = (round + k) % (n2 - 1); b = (round - k + n2 - 1) % (n2 - 1); }
                if (a > b) { const int t = a; a = b; b = t; }
                if (b >= n) continue;              // the padding column is zero
                T* ca = A + a * lda;
                T* cb = A + b * lda;
                T al = 0, be = 0, ga = 0;
                for (int r = lane; r < m; r += 32) {
                    const T x = ca[r], y = cb[r];
                    al += x * x; be += y * y; ga += x * y;
                }
                al = jacobi_warp_sum(al); be = jacobi_warp_sum(be); ga = jacobi_warp_sum(ga);
                if (ga == T(0) || al <= negligible || be <= negligible) continue;
                if (fabs(ga) <= tol * sqrt(al * be)) continue;
                if (lane == 0) *flag = 0;
                const T zeta = (be - al) / (T(2) * ga);
                const T t = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
                const T c = T(1) / sqrt(T(1) + t * t), s = c * t;
                for (int r = lane; r < m; r += 32) {
                    const T x = ca[r], y = cb[r];
                    ca[r] = c * x - s * y;
                    cb[r] = s * x + c * y;
                }
                T* va = V + a * ldv;
                T* vb = V + b * ldv;
                for (int r = lane; r < n; r += 32) {
                    const T x = va[r], y = vb[r];
                    va[r] = c * x - s * y;
                    vb[r] = s * x + c * y;
                }
            }
            __syncthreads();
        }
        const bool done = *flag != 0;
        __syncthreads();
        if (done) break;
    }
}

}  // namespace tn
