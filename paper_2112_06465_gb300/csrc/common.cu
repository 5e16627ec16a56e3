// common.cu -- error reporting, device properties and reduction scratch.
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "hz_internal.cuh"

namespace hz {

static thread_local std::string g_last_error = "no error";

void set_error(const std::string &msg) { g_last_error = msg; }

hz_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    std::string m = std::string(what) + " failed: " + cudaGetErrorString(e) + " (" + file + ":" +
                    std::to_string(line) + ")";
    set_error(m);
    return e == cudaErrorMemoryAllocation ? HZ_ERR_ALLOC : HZ_ERR_CUDA;
}

static std::mutex g_mu;
static std::map<int, DevInfo> g_dev;

hz_status dev_info(DevInfo *out) {
    int dev = 0;
    HZ_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_dev.find(dev);
    if (it == g_dev.end()) {
        DevInfo d;
        d.device = dev;
        HZ_CUDA(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
        HZ_CUDA(cudaDeviceGetAttribute(&d.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
        it = g_dev.emplace(dev, d).first;
    }
    *out = it->second;
    return HZ_OK;
}

// Scratch for single-pass reductions, one per (device, stream).  The
// counter must be zero before every reduction kernel; kernels leave it zero.
static std::map<std::pair<int, cudaStream_t>, RedScratch> g_scratch;

hz_status get_scratch(cudaStream_t s, RedScratch *out) {
    int dev = 0;
    HZ_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, s);
    auto it = g_scratch.find(key);
    if (it == g_scratch.end()) {
        RedScratch r{};
        const size_t bytes = sizeof(double) * kMaxRedBlocks * kMaxRedValues;
        HZ_CUDA(cudaMalloc(&r.partials, bytes));
        HZ_CUDA(cudaMalloc(&r.counter, 256));
        HZ_CUDA(cudaMemset(r.counter, 0, 256));
        HZ_CUDA(cudaDeviceSynchronize());
        it = g_scratch.emplace(key, r).first;
    }
    *out = it->second;
    return HZ_OK;
}

int stream_grid(const DevInfo &d, int64_t work_items, int block, int blocks_per_sm) {
    int64_t need = (work_items + block - 1) / block;
    int64_t cap = (int64_t)d.num_sms * blocks_per_sm;
    if (need < 1) need = 1;
    if (need > cap) need = cap;
    if (need > kMaxRedBlocks) need = kMaxRedBlocks;
    return (int)need;
}

}  // namespace hz

extern "C" HZ_API const char *hz_last_error(void) { return hz::g_last_error.c_str(); }

extern "C" HZ_API int32_t hz_version(void) { return 100; }
