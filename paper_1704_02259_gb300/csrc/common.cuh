// common.cuh -- internal helpers shared by the library's translation units:
// error reporting behind the C ABI, kernel launch accounting, warp helpers
// and the device-side SplitMix64 stream.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "bfs.h"

namespace gbfs {

// Thread-local message behind bfs_last_error().
void set_error(const char *fmt, ...);
void clear_error();

// Launch accounting behind bfs_launch_count().
extern std::atomic<int64_t> g_launches;
inline void count_launch(int k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Returns BFS_OK or records the CUDA error and returns BFS_ERR_CUDA / OOM.
bfs_status cuda_status(cudaError_t e, const char *what, const char *file, int line);

#define GB_CK(call)                                                                  \
    do {                                                                             \
        cudaError_t _e = (call);                                                     \
        if (_e != cudaSuccess) return ::gbfs::cuda_status(_e, #call, __FILE__, __LINE__); \
    } while (0)

// Launch with accounting; checks the launch error.
#define GB_LAUNCH(kernel, grid, block, smem, stream, ...)                            \
    do {                                                                             \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                  \
        ::gbfs::count_launch();                                                      \
        GB_CK(cudaGetLastError());                                                   \
    } while (0)

// Device and pinned host allocations, counted behind bfs_alloc_count() so a
// test can check that a warmed-up (or reserved) path allocates nothing.
extern std::atomic<int64_t> g_allocs;
template <typename T>
inline cudaError_t dev_malloc(T **p, size_t bytes) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
inline cudaError_t dev_malloc_async(T **p, size_t bytes, cudaStream_t st) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocAsync(reinterpret_cast<void **>(p), bytes, st);
}
template <typename T>
inline cudaError_t host_malloc(T **p, size_t bytes, unsigned flags = cudaHostAllocDefault) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaHostAlloc(reinterpret_cast<void **>(p), bytes, flags);
}

// Number of SMs of the current device (cached per device).
int sm_count();

// SplitMix64 (Steele, Lea, Flood 2014): output i of the stream seeded with s
// is the mix13 finaliser applied to s + (i + 1) * 0x9E3779B97F4A7C15.
__host__ __device__ __forceinline__ uint64_t sm64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive prefix sum across the warp; *total receives the warp sum.
__device__ __forceinline__ int warp_exclusive_scan(int v, int *total) {
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane_id() >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x - v;
}

// Loads of data that changes during a traversal. CO (coherent) is set inside
// the persistent kernels, where other blocks wrote the data earlier in the
// same launch: those loads go to L2 (ld.global.cg) instead of the
// non-coherent read-only path.
template <bool CO, typename T>
__device__ __forceinline__ T ld(const T *p) {
    if constexpr (CO) return __ldcg(p);
    else return *p;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (every block resident).
// bar[0] counts arrivals, bar[1] is the generation the last arrival bumps.
// Every wait is bounded: a block that waits longer than timeout_ns sets
// *err, and every block that sees *err leaves; the caller then returns.
// `expected` is gridDim.x except in the self-test, which asks for more.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int32_t *err, unsigned expected,
                             unsigned long long timeout_ns) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *gen = bar + 1;
        volatile int32_t *verr = err;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == expected - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g) {
                if (*verr) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > timeout_ns) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        if (*verr) ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

}  // namespace gbfs
