// Load every kernel of the library into the current device's context up front.
//
// With lazy module loading (the CUDA default) a kernel is loaded on its first
// launch, and loading may synchronise the context.  A request server runs
// long jobs on some streams while it launches short ones on others; a kernel
// variant first used by a short job would then wait for every running job.
// Each translation unit with kernels exposes one of them; through it the
// unit's module is found and all of its functions are loaded (driver entry
// points obtained at run time, so the library needs no link to the driver).
#include <cuda.h>

#include <mutex>
#include <vector>

#include "runtime.h"

namespace tn {

const void* kernels_module_anchor();
const void* tc_module_anchor();
const void* bmps_module_anchor();
const void* ite_module_anchor();

namespace {

template <typename F>
F entry(const char* name) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12040, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return reinterpret_cast<F>(p);
}

}  // namespace

void preload_kernels(int device) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> g(mu);
    for (int d : done)
        if (d == device) return;
    done.push_back(device);
    using GetModule = CUresult (*)(CUmodule*, CUfunction);
    using Count = CUresult (*)(unsigned int*, CUmodule);
    using Enumerate = CUresult (*)(CUfunction*, unsigned int, CUmodule);
    using Load = CUresult (*)(CUfunction);
    const auto get_module = entry<GetModule>("cuFuncGetModule");
    const auto count = entry<Count>("cuModuleGetFunctionCount");
    const auto enumerate = entry<Enumerate>("cuModuleEnumerateFunctions");
    const auto load = entry<Load>("cuFuncLoad");
    if (!get_module || !count || !enumerate || !load) return;   // an older driver: stay lazy
    for (const void* anchor : {kernels_module_anchor(), tc_module_anchor(), bmps_module_anchor(),
                               ite_module_anchor()}) {
        cudaFunction_t f = nullptr;
        if (cudaGetFuncBySymbol(&f, anchor) != cudaSuccess) continue;
        CUmodule mod = nullptr;
        unsigned int n = 0;
        if (get_module(&mod, reinterpret_cast<CUfunction>(f)) != CUDA_SUCCESS || count(&n, mod) != CUDA_SUCCESS)
            continue;
        std::vector<CUfunction> fns(n);
        if (n == 0 || enumerate(fns.data(), n, mod) != CUDA_SUCCESS) continue;
        for (CUfunction fn : fns) load(fn);
    }
    cudaGetLastError();   // a failed query above leaves no sticky error
}

}  // namespace tn
