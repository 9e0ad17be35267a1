// tn_absorb_dot_noalloc: the absorb-dot kernel with its scratch in a fixed,
// file-scope device array instead of memory taken from an allocator.
//
// Who needs this: a caller that must not ask CUDA for memory at the point of
// the call -- for instance a latency-critical loop (cudaMalloc / cudaFree may
// synchronise the whole device and stall every other stream), or a process
// whose device memory is already owned by another allocator (a framework's
// caching allocator, a pre-reserved pool) so that a fresh allocation could fail
// or fragment it.  Such a caller still provides every input and the output.
//
// The array below exists once on every GPU that loads libtn and stays there
// until the process exits.  In host code its name is only a host-side handle,
// so the device address is fetched with cudaGetSymbolAddress the first time a
// device is used (with that device current) and cached per device.
#include <climits>
#include <mutex>

#include "runtime.h"

namespace {

// At most this many tiles of 256 outer positions, i.e. P * S <= 16,777,216.
constexpr long long kNoAllocMaxTiles = 65536;
// 16-byte arrival-counter header followed by one FP64 partial per tile (512 KiB + 16 B).
constexpr size_t kNoAllocBytes = 16 + (size_t)kNoAllocMaxTiles * sizeof(double);
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once).
tn_status scratch_address(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return tn::cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        tn::set_error("device index beyond the fixed-scratch table");
        return TN_ERR_INVALID;
    }
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return tn::cuda_status(e, "cudaGetSymbolAddress(fixed scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return TN_OK;
}

}  // namespace

extern "C" tn_status tn_absorb_dot_noalloc(int dtype, const void* in, const void* E, const void* adj,
                                           int64_t P, int32_t K, int32_t N, int64_t S, double* result,
                                           void* stream) {
    if ((dtype != 0 && dtype != 1) || !in || !E || !adj || !result || P <= 0 || K <= 0 || N <= 0 || S <= 0) {
        tn::set_error("bad absorb-dot arguments");
        return TN_ERR_INVALID;
    }
    if (!tn::absorb_has_fast_path(K, N)) {
        tn::set_error("K, N must be in {1, 4, 16} or {1, 9, 81}");
        return TN_ERR_INVALID;
    }
    // compare without forming P * S, which could overflow for huge arguments
    constexpr long long kMaxOuter = kNoAllocMaxTiles * tn::kAbsorbThreads;   // 16,777,216
    if (P > kMaxOuter / S) {
        tn::set_error("P = " + std::to_string((long long)P) + ", S = " + std::to_string((long long)S) +
                      ": P*S exceeds the 16777216 outer positions the fixed scratch holds");
        return TN_ERR_INVALID;
    }
    const long long tiles = tn::absorb_tiles(P, S, K, N);
    if (tiles > kNoAllocMaxTiles) {
        tn::set_error("more tiles than the fixed scratch holds");
        return TN_ERR_INVALID;
    }
    void* scratch = nullptr;
    tn_status s = scratch_address(&scratch);
    if (s != TN_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The array keeps whatever the previous call left; the arrival counter must start at zero.
    cudaError_t e = cudaMemsetAsync(scratch, 0, 16, st);
    if (e == cudaSuccess) e = tn::launch_absorb_dot_plain(dtype, in, E, adj, P, K, N, S, result, scratch, st);
    return tn::cuda_status(e, "absorb-dot (fixed scratch) launch");
}
