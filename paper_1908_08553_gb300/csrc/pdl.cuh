// Programmatic dependent launch between the grouped launches of a batch run:
// each kernel of the batch path starts by letting the next kernel in the
// stream launch (griddepcontrol.launch_dependents), then waits for the kernel
// before it to finish and flush its memory (griddepcontrol.wait) before it
// reads anything.  The next launch's blocks are thus scheduled while the
// current kernel's last blocks still run, hiding launch latency, and no
// kernel ever reads data its predecessor is still writing.  Launches carry
// the programmatic-stream-serialisation attribute unless the environment sets
// TN_PDL=0 (then every launch waits for its predecessor as usual; the device
// instructions are then no-ops).
#pragma once

#include <cstdlib>
#include <cstring>
#include <utility>

#include <cuda_runtime.h>

namespace tn {

__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

inline bool pdl_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("TN_PDL");
        return !(v && std::strcmp(v, "0") == 0);
    }();
    return on;
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace tn

#define TN_LAUNCH(...)                                  \
    do {                                                \
        const cudaError_t e_l_ = tn::launch_pdl(__VA_ARGS__); \
        if (e_l_ != cudaSuccess) return e_l_;           \
    } while (0)
