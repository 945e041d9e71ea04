// Once-per-device setup of a kernel before its launches.
//
// Raising a kernel's dynamic shared-memory limit (cudaFuncSetAttribute) and
// asking how many of its clusters or blocks can be resident (the occupancy
// calculator) are host-side calls of a few microseconds each.  A served
// stream of small GEMMs launches thousands of kernels per second, so the
// answers are computed once per (kernel, device) and kept.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "launch.h"

namespace tcg {

namespace {
struct Entry {
    cudaError_t err;
    int resident;
};
std::mutex g_mu;
std::map<std::pair<const void*, int>, Entry> g_cache;
}  // namespace

bool pdl_enabled() {
    static const bool on = [] {
        const char* env = getenv("TCGEMM_PDL");
        return !(env && strcmp(env, "0") == 0);
    }();
    return on;
}

cudaError_t kernel_setup(const void* kern, int smem_bytes, const cudaLaunchConfig_t* cluster_cfg, int block_threads,
                         int* resident) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const auto key = std::make_pair(kern, dev);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            if (resident) *resident = it->second.resident;
            return it->second.err;
        }
    }
    Entry en{cudaSuccess, 0};
    if (smem_bytes > 0) en.err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (en.err == cudaSuccess) {
        if (cluster_cfg) {
            if (cudaOccupancyMaxActiveClusters(&en.resident, kern, cluster_cfg) != cudaSuccess) en.resident = 0;
        } else if (block_threads > 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&en.resident, kern, block_threads,
                                                              static_cast<size_t>(smem_bytes)) != cudaSuccess)
                en.resident = 0;
        }
        cudaGetLastError();  // a failed query leaves no sticky error behind
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_cache[key] = en;
    if (resident) *resident = en.resident;
    return en.err;
}

}  // namespace tcg
