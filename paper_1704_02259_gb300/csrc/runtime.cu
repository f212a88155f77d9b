// runtime.cu -- error reporting, launch accounting and device queries behind
// the C ABI (bfs_last_error, bfs_launch_count).
#include <stdarg.h>
#include <stdio.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace gbfs {

std::atomic<int64_t> g_launches{0};
std::atomic<int64_t> g_allocs{0};

static thread_local std::string t_error;

void set_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_error = buf;
}

void clear_error() { t_error.clear(); }

bfs_status cuda_status(cudaError_t e, const char *what, const char *file, int line) {
    const char *base = strrchr(file, '/');
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), base ? base + 1 : file, line);
    if (e == cudaErrorMemoryAllocation) return BFS_ERR_OOM;
    return BFS_ERR_CUDA;
}

int sm_count() {
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (cache[dev] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 1;
        cache[dev] = v;
    }
    return cache[dev];
}

}  // namespace gbfs

extern "C" BFS_API const char *bfs_last_error(void) { return gbfs::t_error.c_str(); }

extern "C" BFS_API int64_t bfs_launch_count(void) {
    return gbfs::g_launches.load(std::memory_order_relaxed);
}

extern "C" BFS_API int64_t bfs_alloc_count(void) {
    return gbfs::g_allocs.load(std::memory_order_relaxed);
}
