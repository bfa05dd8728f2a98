// Persistent-grid sizing: resident blocks per SM times the SM count, cached
// per (device, kernel, block size, shared memory).
#include <map>
#include <mutex>
#include <tuple>

#include "lbrd_kernels.h"

namespace lbrd {

namespace {
std::mutex g_mu;
std::map<std::tuple<int, const void *, int, size_t>, unsigned> g_cache;
std::map<int, int> g_sms;

int sm_count_locked(int dev) {
    auto it = g_sms.find(dev);
    if (it != g_sms.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    g_sms[dev] = n;
    return n;
}
}  // namespace

unsigned occupancy_blocks(const void *kernel, int nthreads, size_t smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_mu);
    const auto key = std::make_tuple(dev, kernel, nthreads, smem);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nthreads, smem) != cudaSuccess || per_sm <= 0)
        per_sm = 1;
    const unsigned blocks = (unsigned)per_sm * (unsigned)sm_count_locked(dev);
    g_cache[key] = blocks;
    return blocks;
}

unsigned max_persistent_blocks() {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_mu);
    return 32u * (unsigned)sm_count_locked(dev);  // at most 32 resident blocks per SM
}

}  // namespace lbrd
