// gen.cu -- graph input on the GPU: the R-MAT / Kronecker edge generator and
// its Erdos-Renyi control (Sec. 6.2), the symmetric CSR builder (Sec. 6.2
// "bidirectional" edges, Sec. 6.3 CSR), and the seeded root sampler (Sec. 6.3).
//
// CSR build = keys (src << B | dst, both directions, self-loops mapped to a
// sentinel) -> stable LSD radix sort with 8-bit digits -> order-preserving
// compaction of the first copy of every key, which writes the indices and,
// at every row start, the offsets.
#include <stdio.h>

#include "common.cuh"

namespace gbfs {

namespace {

constexpr uint64_t kPermBase = 1ull << 62;

struct Perm {
    uint64_t a[3];
    uint64_t c[3];
    uint64_t mask;
    int h;
};

Perm make_perm(int scale, uint64_t seed) {
    Perm p;
    for (int j = 0; j < 3; ++j) {
        p.a[j] = sm64_at(seed, kPermBase + 2ull * j) | 1ull;
        p.c[j] = sm64_at(seed, kPermBase + 2ull * j + 1ull);
    }
    p.mask = (1ull << scale) - 1ull;
    p.h = (scale + 1) / 2;
    return p;
}

// Seeded bijection of [0, 2^scale): three rounds of (odd affine map mod
// 2^scale, then x ^= x >> ceil(scale/2)); every round is invertible.
__device__ __forceinline__ uint32_t relabel(uint32_t x, const Perm &p) {
    uint64_t y = x;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        y = (y * p.a[j] + p.c[j]) & p.mask;
        y ^= y >> p.h;
    }
    return (uint32_t)y;
}

// One thread per edge (grid-stride). Bit level b of edge e takes the high
// half of SplitMix64 output e*scale+b and picks quadrant
// [0,t1) -> (0,0), [t1,t2) -> (0,1), [t2,t3) -> (1,0), [t3,2^32) -> (1,1).
__global__ void gen_rmat_kernel(int scale, uint64_t seed, uint64_t t1, uint64_t t2, uint64_t t3,
                                Perm perm, int64_t m, int32_t *__restrict__ src,
                                int32_t *__restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t s = 0, d = 0;
        uint64_t base = (uint64_t)e * (uint64_t)scale;
        for (int lev = 0; lev < scale; ++lev) {
            uint64_t u = sm64_at(seed, base + lev) >> 32;
            uint32_t sbit = u >= t2;
            uint32_t dbit = (u >= t1 && u < t2) || u >= t3;
            s |= sbit << lev;
            d |= dbit << lev;
        }
        src[e] = (int32_t)relabel(s, perm);
        dst[e] = (int32_t)relabel(d, perm);
    }
}

__global__ void gen_er_kernel(int scale, uint64_t seed, int64_t m, int32_t *__restrict__ src,
                              int32_t *__restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        src[e] = (int32_t)(sm64_at(seed, 2ull * e) >> (64 - scale));
        dst[e] = (int32_t)(sm64_at(seed, 2ull * e + 1ull) >> (64 - scale));
    }
}

// ------------------------------------------------------------------ CSR
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 16;
constexpr int kRsTile = kRsThreads * kRsItems;  // keys per tile
constexpr int kRsRadix = 256;

__global__ void make_keys_kernel(int64_t m, const int32_t *__restrict__ src,
                                 const int32_t *__restrict__ dst, int64_t n, int B,
                                 uint64_t sentinel, ulonglong2 *__restrict__ keys,
                                 int *__restrict__ bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = src[e], d = dst[e];
        ulonglong2 k;
        if (s < 0 || s >= n || d < 0 || d >= n) {
            *bad = 1;
            k.x = k.y = sentinel;
        } else if (s == d) {
            k.x = k.y = sentinel;  // self-loops are dropped
        } else {
            k.x = ((uint64_t)s << B) | (uint64_t)d;
            k.y = ((uint64_t)d << B) | (uint64_t)s;
        }
        keys[e] = k;
    }
}

// Digit histogram of each block's contiguous key range: counts[digit * G + b].
__global__ void __launch_bounds__(kRsThreads) rs_hist_kernel(const uint64_t *__restrict__ keys,
                                                             int64_t N, int64_t per_block,
                                                             int shift, uint32_t *counts) {
    __shared__ uint32_t h[kRsRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t beg = blockIdx.x * per_block;
    int64_t end = min(N, beg + per_block);
    for (int64_t i = beg + threadIdx.x; i < end; i += kRsThreads)
        atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
    __syncthreads();
    counts[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `len` uint32 counts into uint64 out[0..len); out[len] =
// total. One block of 1024 threads walks the array in chunks.
__global__ void __launch_bounds__(1024) scan_u32_kernel(const uint32_t *__restrict__ in,
                                                        int64_t len, uint64_t *__restrict__ out) {
    __shared__ unsigned long long warp_tot[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < len; base += 1024) {
        int64_t i = base + threadIdx.x;
        unsigned long long v = i < len ? in[i] : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            unsigned long long t = warp_tot[lane];
            unsigned long long s = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
                if ((int)lane >= o) s += y;
            }
            warp_tot[lane] = s - t;  // exclusive warp offsets
        }
        __syncthreads();
        unsigned long long excl = carry + warp_tot[wid] + x - v;
        if (i < len) out[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[len] = carry;
}

// Stable scatter of one 8-bit digit. Block b owns the contiguous range
// [b*per_block, ...) and walks it in tiles of kRsTile keys, in order. Inside
// a tile warp w owns 512 consecutive keys, read 32 at a time in order; equal
// digits within a round are ranked with __match_any_sync, and per-warp digit
// counters carry the rank across rounds. Warps are then ordered by a prefix
// over the 8 counters of each digit, which keeps the sort stable.
__global__ void __launch_bounds__(kRsThreads) rs_scatter_kernel(
    const uint64_t *__restrict__ in, uint64_t *__restrict__ out, int64_t N, int64_t per_block,
    int shift, const uint64_t *__restrict__ offs) {
    __shared__ uint32_t wcnt[kRsWarps][kRsRadix];
    __shared__ unsigned long long dbase[kRsRadix];
    __shared__ uint32_t ttot[kRsRadix];
    const unsigned tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t beg = blockIdx.x * per_block;
    const int64_t end = min(N, beg + per_block);
    dbase[tid] = offs[(int64_t)tid * gridDim.x + blockIdx.x];
    const unsigned lt = lanemask_lt();
    for (int64_t t = beg; t < end; t += kRsTile) {
#pragma unroll
        for (int i = 0; i < kRsWarps; ++i) wcnt[i][tid] = 0;
        __syncthreads();
        uint64_t k[kRsItems];
        uint32_t rk[kRsItems];
#pragma unroll
        for (int r = 0; r < kRsItems; ++r) {
            int64_t idx = t + (int64_t)w * (32 * kRsItems) + r * 32 + lane;
            bool valid = idx < end;
            uint64_t key = valid ? in[idx] : 0ull;
            unsigned dig = valid ? (unsigned)((key >> shift) & 255u) : 256u + lane;
            unsigned peers = __match_any_sync(0xffffffffu, dig);
            unsigned lower = __popc(peers & lt);
            uint32_t cb = valid ? wcnt[w][dig] : 0u;
            __syncwarp();
            if (valid && lower == 0) wcnt[w][dig] = cb + __popc(peers);
            __syncwarp();
            k[r] = key;
            rk[r] = cb + lower;
        }
        __syncthreads();
        {
            uint32_t run = 0;
#pragma unroll
            for (int i = 0; i < kRsWarps; ++i) {
                uint32_t c = wcnt[i][tid];
                wcnt[i][tid] = run;
                run += c;
            }
            ttot[tid] = run;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRsItems; ++r) {
            int64_t idx = t + (int64_t)w * (32 * kRsItems) + r * 32 + lane;
            if (idx < end) {
                unsigned dig = (unsigned)((k[r] >> shift) & 255u);
                out[dbase[dig] + wcnt[w][dig] + rk[r]] = k[r];
            }
        }
        __syncthreads();
        dbase[tid] += ttot[tid];
        __syncthreads();
    }
}

// Number of first copies of non-sentinel keys per tile of kRsTile keys.
__global__ void __launch_bounds__(kRsThreads) uniq_count_kernel(const uint64_t *__restrict__ keys,
                                                                int64_t N, uint64_t sentinel,
                                                                uint32_t *__restrict__ counts) {
    __shared__ uint32_t wsum[kRsWarps];
    int64_t t0 = (int64_t)blockIdx.x * kRsTile;
    uint32_t c = 0;
    for (int j = 0; j < kRsItems; ++j) {
        int64_t i = t0 + j * kRsThreads + threadIdx.x;
        if (i < N) {
            uint64_t k = keys[i];
            c += (k != sentinel && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
        }
    }
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int i = 0; i < kRsWarps; ++i) s += wsum[i];
        counts[blockIdx.x] = s;
    }
}

// Order-preserving compaction: thread t of tile b owns keys
// [b*kRsTile + 16t, +16). Writes indices[pos] = dst of every first copy and,
// where a row starts, offsets[v] = pos for every v since the previous row
// (degree-0 vertices included). The thread holding the last non-sentinel key
// fills offsets[s+1 .. n] with nnz = tile_offs[ntiles].
__global__ void __launch_bounds__(kRsThreads) uniq_write_kernel(
    const uint64_t *__restrict__ keys, int64_t N, uint64_t sentinel, int B, int64_t n,
    const uint64_t *__restrict__ tile_offs, int64_t ntiles, int32_t *__restrict__ indices,
    int64_t *__restrict__ offsets) {
    __shared__ uint32_t wsum[kRsWarps];
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t i0 = (int64_t)blockIdx.x * kRsTile + (int64_t)threadIdx.x * kRsItems;
    uint32_t c = 0;
    for (int j = 0; j < kRsItems; ++j) {
        int64_t i = i0 + j;
        if (i < N) {
            uint64_t k = keys[i];
            c += (k != sentinel && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
        }
    }
    int tot;
    int excl = warp_exclusive_scan((int)c, &tot);
    if (lane == 31) wsum[w] = (uint32_t)tot;
    __syncthreads();
    uint64_t base = tile_offs[blockIdx.x];
    for (unsigned i = 0; i < w; ++i) base += wsum[i];
    base += (uint64_t)excl;
    const uint64_t nnz = tile_offs[ntiles];
    const uint64_t dmask = (1ull << B) - 1ull;
    for (int j = 0; j < kRsItems; ++j) {
        int64_t i = i0 + j;
        if (i >= N) break;
        uint64_t k = keys[i];
        if (k == sentinel) break;  // sentinels sort last
        int64_t s = (int64_t)(k >> B);
        uint64_t prev = i > 0 ? keys[i - 1] : 0ull;
        bool first = (i == 0 || prev != k);
        if (first) {
            indices[base] = (int32_t)(k & dmask);
            int64_t ps = i > 0 ? (int64_t)(prev >> B) : -1;
            for (int64_t v = ps + 1; v <= s; ++v) offsets[v] = (int64_t)base;
            ++base;
        }
        bool last = (i + 1 == N) || keys[i + 1] == sentinel;
        if (last)
            for (int64_t v = s + 1; v <= n; ++v) offsets[v] = (int64_t)nnz;
    }
}

__global__ void __launch_bounds__(256) sample_roots_kernel(const int64_t *__restrict__ off,
                                                           int64_t n, uint64_t seed, int k,
                                                           int64_t max_draws,
                                                           int32_t *__restrict__ roots,
                                                           int32_t *__restrict__ count) {
    __shared__ int32_t chosen[4096];
    __shared__ int32_t cand[256];
    __shared__ int got;
    if (threadIdx.x == 0) got = 0;
    __syncthreads();
    for (int64_t base = 0; base < max_draws; base += 256) {
        if (got >= k) break;
        int64_t j = base + threadIdx.x;
        int32_t r = -1;
        if (j < max_draws) {
            int64_t rr = (int64_t)(sm64_at(seed, (uint64_t)j) % (uint64_t)n);
            if (off[rr + 1] - off[rr] >= 1) r = (int32_t)rr;
        }
        cand[threadIdx.x] = r;
        __syncthreads();
        for (int t = 0; t < 256; ++t) {
            int32_t c = cand[t];
            if (c < 0) continue;
            if (got >= k) break;
            int dup = 0;
            for (int i = threadIdx.x; i < got; i += 256) dup |= (chosen[i] == c);
            dup = __syncthreads_or(dup);
            if (!dup && threadIdx.x == 0) {
                chosen[got] = c;
                got = got + 1;
            }
            __syncthreads();
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < got; i += 256) roots[i] = chosen[i];
    if (threadIdx.x == 0) *count = got;
}

int grid_for(int64_t work, int threads, int per_sm = 8) {
    int64_t g = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace
}  // namespace gbfs

using namespace gbfs;

extern "C" BFS_API bfs_status bfs_generate_edges(int32_t kind, int32_t scale, int32_t edgefactor,
                                                 uint64_t seed, double a, double b, double c,
                                                 int32_t *src, int32_t *dst, void *stream) {
    clear_error();
    if (kind != BFS_GEN_RMAT && kind != BFS_GEN_ER) {
        set_error("bfs_generate_edges: unknown kind %d", kind);
        return BFS_ERR_INVALID;
    }
    if (scale < 1 || scale > 30 || edgefactor < 1 || edgefactor > 1024 || !src || !dst) {
        set_error("bfs_generate_edges: need 1<=scale<=30, 1<=edgefactor<=1024, non-null outputs");
        return BFS_ERR_INVALID;
    }
    if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) {
        set_error("bfs_generate_edges: initiator probabilities must be >= 0 and sum to <= 1");
        return BFS_ERR_INVALID;
    }
    int64_t m = (int64_t)edgefactor << scale;
    cudaStream_t st = as_stream(stream);
    int grid = grid_for(m, 256, 16);
    if (kind == BFS_GEN_RMAT) {
        uint64_t t1 = (uint64_t)(a * 4294967296.0);
        uint64_t t2 = (uint64_t)((a + b) * 4294967296.0);
        uint64_t t3 = (uint64_t)((a + b + c) * 4294967296.0);
        GB_LAUNCH(gen_rmat_kernel, grid, 256, 0, st, scale, seed, t1, t2, t3,
                  make_perm(scale, seed), m, src, dst);
    } else {
        GB_LAUNCH(gen_er_kernel, grid, 256, 0, st, scale, seed, m, src, dst);
    }
    return BFS_OK;
}

namespace {
struct AsyncBuf {
    void *p = nullptr;
    cudaStream_t st;
    explicit AsyncBuf(cudaStream_t s) : st(s) {}
    cudaError_t alloc(size_t bytes) { return dev_malloc_async(&p, bytes ? bytes : 16, st); }
    ~AsyncBuf() {
        if (p) cudaFreeAsync(p, st);
    }
};
}  // namespace

extern "C" BFS_API bfs_status bfs_build_csr(int64_t n, int64_t m, const int32_t *src,
                                            const int32_t *dst, int64_t *offsets,
                                            int32_t *indices, int64_t *nnz_out, void *stream) {
    clear_error();
    if (n < 1 || n >= (1ll << 31) || m < 0 || m > (1ll << 32) || !offsets || !nnz_out ||
        (m > 0 && (!src || !dst || !indices))) {
        set_error("bfs_build_csr: need 1 <= n < 2^31, 0 <= m <= 2^32 and non-null buffers");
        return BFS_ERR_INVALID;
    }
    cudaStream_t st = as_stream(stream);
    if (m == 0) {
        GB_CK(cudaMemsetAsync(offsets, 0, (size_t)(n + 1) * sizeof(int64_t), st));
        GB_CK(cudaStreamSynchronize(st));
        *nnz_out = 0;
        return BFS_OK;
    }
    int B = 1;
    while ((1ll << B) < n) ++B;
    const uint64_t sentinel = (1ull << (2 * B)) - 1ull;
    const int64_t N = 2 * m;

    // Radix-sort geometry: G blocks, each a contiguous multiple of kRsTile keys.
    int occ = 0;
    GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, rs_scatter_kernel, kRsThreads, 0));
    if (occ < 1) occ = 1;
    int64_t tiles = (N + kRsTile - 1) / kRsTile;
    int64_t G = std::min<int64_t>(tiles, (int64_t)sm_count() * occ);
    int64_t per_block = ((tiles + G - 1) / G) * kRsTile;
    G = (N + per_block - 1) / per_block;

    AsyncBuf ka(st), kb(st), cnt(st), offs(st), tcnt(st), toffs(st), bad(st);
    GB_CK(ka.alloc((size_t)N * 8));
    GB_CK(kb.alloc((size_t)N * 8));
    GB_CK(cnt.alloc((size_t)kRsRadix * G * 4));
    GB_CK(offs.alloc((size_t)(kRsRadix * G + 1) * 8));
    GB_CK(tcnt.alloc((size_t)tiles * 4));
    GB_CK(toffs.alloc((size_t)(tiles + 1) * 8));
    GB_CK(bad.alloc(sizeof(int)));
    GB_CK(cudaMemsetAsync(bad.p, 0, sizeof(int), st));

    uint64_t *kin = (uint64_t *)ka.p, *kout = (uint64_t *)kb.p;
    GB_LAUNCH(make_keys_kernel, grid_for(m, 256, 16), 256, 0, st, m, src, dst, n, B, sentinel,
              (ulonglong2 *)kin, (int *)bad.p);
    const int passes = (2 * B + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        GB_LAUNCH(rs_hist_kernel, (int)G, kRsThreads, 0, st, kin, N, per_block, shift,
                  (uint32_t *)cnt.p);
        GB_LAUNCH(scan_u32_kernel, 1, 1024, 0, st, (const uint32_t *)cnt.p, kRsRadix * G,
                  (uint64_t *)offs.p);
        GB_LAUNCH(rs_scatter_kernel, (int)G, kRsThreads, 0, st, kin, kout, N, per_block, shift,
                  (const uint64_t *)offs.p);
        std::swap(kin, kout);
    }
    GB_LAUNCH(uniq_count_kernel, (int)tiles, kRsThreads, 0, st, kin, N, sentinel,
              (uint32_t *)tcnt.p);
    GB_LAUNCH(scan_u32_kernel, 1, 1024, 0, st, (const uint32_t *)tcnt.p, tiles,
              (uint64_t *)toffs.p);
    GB_LAUNCH(uniq_write_kernel, (int)tiles, kRsThreads, 0, st, kin, N, sentinel, B, n,
              (const uint64_t *)toffs.p, tiles, indices, offsets);
    int64_t nnz = 0;
    int hbad = 0;
    GB_CK(cudaMemcpyAsync(&nnz, (uint64_t *)toffs.p + tiles, 8, cudaMemcpyDeviceToHost, st));
    GB_CK(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GB_CK(cudaStreamSynchronize(st));
    if (hbad) {
        set_error("bfs_build_csr: an edge endpoint is outside [0, %lld)", (long long)n);
        return BFS_ERR_INVALID;
    }
    if (nnz == 0) {
        GB_CK(cudaMemsetAsync(offsets, 0, (size_t)(n + 1) * sizeof(int64_t), st));
        GB_CK(cudaStreamSynchronize(st));
    }
    *nnz_out = nnz;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_sample_roots(const int64_t *offsets, int64_t n, uint64_t seed,
                                               int32_t k, int64_t max_draws, int32_t *roots_out,
                                               int32_t *count_out, void *stream) {
    clear_error();
    if (!offsets || !roots_out || !count_out || n < 1 || n >= (1ll << 31) || k < 1 ||
        k > 4096 || max_draws < 1) {
        set_error("bfs_sample_roots: need offsets, outputs, 1 <= n < 2^31, 1 <= k <= 4096");
        return BFS_ERR_INVALID;
    }
    cudaStream_t st = as_stream(stream);
    AsyncBuf dcount(st);
    GB_CK(dcount.alloc(sizeof(int32_t)));
    GB_LAUNCH(sample_roots_kernel, 1, 256, 0, st, offsets, n, seed, k, max_draws, roots_out,
              (int32_t *)dcount.p);
    int32_t got = 0;
    GB_CK(cudaMemcpyAsync(&got, dcount.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GB_CK(cudaStreamSynchronize(st));
    *count_out = got;
    return BFS_OK;
}
