// msbfs.cu -- batched multi-source BFS: up to 512 roots share one traversal.
//
// Root i owns bit i of a per-vertex bitset of W 64-bit words (W = 1, 2, 4 or
// 8): seen[v] (roots that reached v) and, per layer j, the frontier words
// fr_j[v] (roots that reached v at distance exactly j). A layer is
//   bottom-up (Alg. 2 on bit lanes): every vertex still lacking some live
//     root ORs the frontier words of its neighbours, in CSR order, and stops
//     as soon as every lacking root is found -- the paper's early exit, taken
//     per lane set. A lane scans `lane_probe` neighbours alone; longer rows
//     are finished by the warp with a 64-bit OR reduction over 32 neighbours
//     per round;
//   top-down (Alg. 1 on bit lanes): the vertices holding frontier bits are
//     compacted into a list (heavy ones into a grid-spread list), their
//     frontier words are ORed into each neighbour's next words with 64-bit
//     atomicOr, and a dense pass keeps the bits not yet seen.
// A root whose frontier is empty has finished; it leaves the live-lane mask
// (the OR of the layer's new bits), so no vertex waits for it any longer and
// the early exit stays effective when some roots sit in small components.
// The direction is the edge form of the Alg. 3 switch over vertex counts:
// e_f is the degree sum of vertices holding a frontier bit, e_u that of
// vertices still lacking some live root.
//
// Levels are not written per layer: the frontier words of every layer stay
// in a ring of `lcap` slots, and one pass at the end turns them into the
// int8 level rows, a warp storing 32 consecutive bytes of a row per
// instruction (whole sectors, -1 where no layer holds the bit). Should a
// traversal need more layers than slots, the full slots are turned into
// levels the same way before the ring wraps, and later layers write only
// their reached pairs.

#include <stdio.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>

#include "graph.cuh"

struct MsState {
    int W = 0;     // lane words the bitsets are sized for
    int lcap = 0;  // frontier slots
    int64_t n = 0;
    unsigned long long *seen = nullptr;  // [n][W]
    unsigned long long *fr = nullptr;    // [lcap][n][W]; layer j in slot j % lcap
    unsigned long long *live = nullptr;  // [3][8] live-lane masks, ring by layer
    int32_t *list = nullptr, *big = nullptr, *roots = nullptr;
    int64_t *trace = nullptr;
    int64_t *h_slot = nullptr;  // pinned: one trace slot (8) and one live mask (8)
    // mapped pinned block polled by the host loop: slot (8), live mask (8),
    // sequence number; d_pub is its device address
    int64_t *h_pub = nullptr, *d_pub = nullptr;
    int64_t pub_seq = 0;
    bfs_batch_config cfg;
    std::vector<bfs_batch_layer_stats> last;
    int64_t last_pairs = 0;
    std::vector<cudaEvent_t> events;
    // device-loop variant: control block (layer records, result, barrier)
    // and the captured graph with the arguments it was captured for
    int64_t *pctl = nullptr, *h_pctl = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;  // private stream the graph is captured on
    int g_W = 0, g_k = -1;
    const void *g_levels = nullptr, *g_seen = nullptr;
    bfs_batch_config g_cfg;
};

namespace gbfs {

void free_ms_state(bfs_graph *g) {
    if (!g || !g->ms) return;
    MsState *m = g->ms;
    cudaFree(m->seen);
    cudaFree(m->fr);
    cudaFree(m->live);
    cudaFree(m->list);
    cudaFree(m->big);
    cudaFree(m->roots);
    cudaFree(m->trace);
    cudaFree(m->pctl);
    if (m->h_slot) cudaFreeHost(m->h_slot);
    if (m->h_pub) cudaFreeHost(m->h_pub);
    if (m->h_pctl) cudaFreeHost(m->h_pctl);
    if (m->exec) cudaGraphExecDestroy(m->exec);
    if (m->graph) cudaGraphDestroy(m->graph);
    if (m->cap) cudaStreamDestroy(m->cap);
    for (cudaEvent_t e : m->events) cudaEventDestroy(e);
    delete m;
    g->ms = nullptr;
}

namespace {

// Trace slot fields; the step kernels add fields 0-5 with one block_add.
//   M_NV, M_MF      vertices holding a bit of the new frontier, degree sum
//   M_PAIRS         (root, vertex) pairs of the new frontier
//   M_LACKN/DEG     vertices (degree >= 1) still lacking some live root after
//                   the layer, degree sum (the next layer's v_u, e_u)
//   M_EXAM          edges examined
//   M_LIST, M_BIG   top-down compaction counts (of the slot's own layer)
enum MsField { M_NV = 0, M_MF = 1, M_PAIRS = 2, M_LACKN = 3, M_LACKDEG = 4, M_EXAM = 5,
               M_LIST = 6, M_BIG = 7 };
constexpr int kMsBlock = 256;
constexpr int kMsBigBatch = 1024;
constexpr int kMaxRoots = 512;
constexpr int kMaxSlots = 16;
constexpr int kPctlLayers = 128;  // layer records of the device loop (depth <= 127)

template <int W>
struct Lanes {
    unsigned long long w[W];
};

template <int W, bool CO>
__device__ __forceinline__ void load_lanes(const unsigned long long *p,
                                           unsigned long long (&x)[W]) {
    if constexpr (W == 1) {
        x[0] = CO ? __ldcg(p) : __ldg(p);
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2) {
            const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(p) + i / 2;
            const ulonglong2 t = CO ? __ldcg(q) : __ldg(q);
            x[i] = t.x;
            x[i + 1] = t.y;
        }
    }
}

template <int W>
__device__ __forceinline__ Lanes<W> load_live(const unsigned long long *p) {
    Lanes<W> a;
#pragma unroll
    for (int i = 0; i < W; ++i) a.w[i] = __ldcg(p + i);
    return a;
}

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)x);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// Sums the 6 step counters over the block and adds them to dst[0..6), and
// ORs the block's new bits into the next live mask: one atomic per counter
// and lane word.
template <int W>
__device__ __forceinline__ void block_finish(int64_t (&v)[6], const unsigned long long (&nb)[W],
                                             unsigned long long *dst,
                                             unsigned long long *live_next) {
    __shared__ long long red[6][kMsBlock / 32];
    __shared__ unsigned long long lv[W];
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x < W) lv[threadIdx.x] = 0ull;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int64_t s = warp_sum(v[i]);
        if (lane == 0) red[i][w] = s;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const unsigned long long x = warp_or64(nb[i]);
        if (lane == 0 && x) atomicOr(lv + i, x);
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        long long s = 0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += red[threadIdx.x][j];
        if (s) atomicAdd(dst + threadIdx.x, (unsigned long long)s);
    }
    if (threadIdx.x < W && lv[threadIdx.x]) atomicOr(live_next + threadIdx.x, lv[threadIdx.x]);
}

// seen = 0 and the first frontier slot = 0.
__global__ void ms_fill_kernel(unsigned long long *__restrict__ seen,
                               unsigned long long *__restrict__ fr0, int64_t nwords) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nwords; i += stride) {
        seen[i] = 0ull;
        fr0[i] = 0ull;
    }
}

// Roots: lane l sets bit l of its root's seen and frontier words. Slot 0 of
// the trace gets the first frontier's counters (distinct root vertices, their
// degrees, pairs = k, and the vertices of degree >= 1 still lacking a root:
// all of them but the root vertices that every root starts from). The live
// mask ring starts as the k lanes.
template <int W>
__global__ void __launch_bounds__(kMaxRoots) ms_roots_kernel(
    const int32_t *__restrict__ roots, int k, int64_t n, int64_t nondeg0, int64_t nnz,
    const int64_t *__restrict__ off, Lanes<W> act, unsigned long long *__restrict__ seen,
    unsigned long long *__restrict__ fr0, unsigned long long *__restrict__ live,
    int64_t *__restrict__ trace) {
    __shared__ long long red[5][kMaxRoots / 32];
    const int l = threadIdx.x;
    if (l < k) {
        const int64_t v = roots[l];
        atomicOr(seen + v * W + (l >> 6), 1ull << (l & 63));
        atomicOr(fr0 + v * W + (l >> 6), 1ull << (l & 63));
    }
    if (l < 8) {
        live[l] = l < W ? act.w[l] : 0ull;
        live[8 + l] = 0ull;
        live[16 + l] = 0ull;
    }
    __syncthreads();
    int64_t c[5] = {0, 0, 0, 0, 0};
    if (l < k) {
        const int32_t v = roots[l];
        bool first = true;
        for (int j = 0; j < l; ++j) first = first && roots[j] != v;
        if (first) {
            const int64_t d = off[v + 1] - off[v];
            c[0] = 1;
            c[1] = d;
            bool full = true;
#pragma unroll
            for (int i = 0; i < W; ++i) full = full && seen[(int64_t)v * W + i] == act.w[i];
            if (full && d > 0) {
                c[3] = 1;
                c[4] = d;
            }
        }
    }
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int64_t s = warp_sum(c[i]);
        if (lane == 0) red[i][w] = s;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        long long s = 0;
        if (threadIdx.x < 5)
            for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += red[threadIdx.x][j];
        long long out = s;
        if (threadIdx.x == M_PAIRS) out = k;
        if (threadIdx.x == M_LACKN) out = nondeg0 - s;
        if (threadIdx.x == M_LACKDEG) out = nnz - s;
        if (threadIdx.x >= 5) out = 0;
        trace[threadIdx.x] = out;
    }
}

// Records the newly reached bits `nw` of vertex v (degree deg >= 1): seen,
// counters, the block's live OR; and counts v as lacking when some live
// root has still not reached it.
template <int W>
__device__ __forceinline__ void ms_commit(int64_t v, int64_t deg,
                                          const unsigned long long (&s)[W],
                                          const unsigned long long (&nw)[W], const Lanes<W> &act,
                                          unsigned long long *__restrict__ seen, int64_t (&c)[6],
                                          unsigned long long (&nb)[W]) {
    bool any = false, lacking = false;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        any = any || nw[i] != 0ull;
        lacking = lacking || (act.w[i] & ~(s[i] | nw[i])) != 0ull;
    }
    if (any) {
#pragma unroll
        for (int i = 0; i < W; ++i) {
            if (!nw[i]) continue;
            seen[v * W + i] = s[i] | nw[i];
            c[2] += __popcll(nw[i]);
            nb[i] |= nw[i];
        }
        c[0] += 1;
        c[1] += deg;
    }
    if (lacking) {
        c[3] += 1;
        c[4] += deg;
    }
}

// Bottom-up layer on bit lanes. Warp per 32 consecutive vertices, lane per
// vertex. need = live roots this vertex still lacks; acc = OR of the
// neighbours' frontier words restricted to need, in CSR order, stopping once
// acc = need. acc is the vertex's next-frontier word set (written for every
// vertex, so the next slot needs no clearing).
template <int W, bool CO>
__device__ __forceinline__ void ms_bu_phase(
    const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
    const uint32_t *__restrict__ base_vis, int64_t n, Lanes<W> act,
    unsigned long long *__restrict__ seen, const unsigned long long *__restrict__ cur,
    unsigned long long *__restrict__ nxt, int probe, unsigned long long *slot_next,
    int64_t *zero_slot, unsigned long long *live_next, unsigned long long *live_zero) {
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        zero_slot[threadIdx.x] = 0;
        live_zero[threadIdx.x] = 0ull;
    }
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nwords = (n + 31) / 32;
    int64_t c[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long nb[W];
#pragma unroll
    for (int i = 0; i < W; ++i) nb[i] = 0ull;
    for (int64_t w = gw; w < nwords; w += tw) {
        const int64_t v = w * 32 + lane;
        const bool inb = v < n;
        const uint32_t bw = base_vis[w];
        const bool skip = !inb || ((bw >> lane) & 1u);  // degree 0 or past n
        unsigned long long s[W], need[W], acc[W];
        bool anyneed = false;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            s[i] = skip ? 0ull : ld<CO>(seen + v * W + i);
            need[i] = skip ? 0ull : (act.w[i] & ~s[i]);
            acc[i] = 0ull;
            anyneed = anyneed || need[i] != 0ull;
        }
        int64_t beg = 0, end = 0;
        bool done = !anyneed;
        int64_t ex = 0;
        if (!done) {
            beg = off[v];
            end = off[v + 1];
            const int64_t lim = min(end - beg, (int64_t)probe);
            for (int64_t q = 0; q < lim; ++q) {
                const int64_t u = __ldg(idx + beg + q);
                unsigned long long x[W];
                load_lanes<W, CO>(cur + u * W, x);
                ++ex;
                bool comp = true;
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    acc[i] |= x[i] & need[i];
                    comp = comp && acc[i] == need[i];
                }
                if (comp) {
                    done = true;
                    break;
                }
            }
        }
        unsigned pend = __ballot_sync(0xffffffffu, !done && end - beg > probe);
        while (pend) {
            const int L = __ffs(pend) - 1;
            pend &= pend - 1;
            const int64_t lb = __shfl_sync(0xffffffffu, beg + probe, L);
            const int64_t le = __shfl_sync(0xffffffffu, end, L);
            unsigned long long nL[W], aL[W];
#pragma unroll
            for (int i = 0; i < W; ++i) {
                nL[i] = __shfl_sync(0xffffffffu, need[i], L);
                aL[i] = __shfl_sync(0xffffffffu, acc[i], L);
            }
            int64_t exL = 0;
            for (int64_t e0 = lb; e0 < le; e0 += 32) {
                const int64_t e = e0 + lane;
                unsigned long long x[W];
                if (e < le) {
                    const int64_t u = __ldg(idx + e);
                    load_lanes<W, CO>(cur + u * W, x);
                } else {
#pragma unroll
                    for (int i = 0; i < W; ++i) x[i] = 0ull;
                }
                bool comp = true;
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    aL[i] |= warp_or64(x[i] & nL[i]);
                    comp = comp && aL[i] == nL[i];
                }
                exL += min((int64_t)32, le - e0);
                if (comp) break;
            }
            if ((int)lane == L) {
#pragma unroll
                for (int i = 0; i < W; ++i) acc[i] = aL[i];
                ex += exL;
            }
        }
        if (inb) {
#pragma unroll
            for (int i = 0; i < W; ++i) nxt[v * W + i] = acc[i];
            if (!skip) ms_commit<W>(v, end - beg, s, acc, act, seen, c, nb);
        }
        c[5] += ex;
    }
    block_finish<W>(c, nb, slot_next, live_next);
}

// Vertices holding a frontier bit -> list (block scan, one atomic per
// block); those of degree >= big_deg -> the grid-spread list instead.
template <int W, bool CO>
__device__ __forceinline__ void ms_compact_phase(
    const unsigned long long *__restrict__ cur, int64_t n, const int64_t *__restrict__ off,
    int64_t big_deg, int32_t *__restrict__ list, int32_t *__restrict__ big,
    unsigned long long *slot_cur) {
    __shared__ int wtot[kMsBlock / 32];
    __shared__ unsigned long long base_s;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    constexpr int per = 4;
    for (int64_t t0 = (int64_t)blockIdx.x * kMsBlock * per; t0 < n;
         t0 += (int64_t)gridDim.x * kMsBlock * per) {
        const int64_t v0 = t0 + (int64_t)threadIdx.x * per;
        bool small[per];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < per; ++k) {
            const int64_t v = v0 + k;
            bool active = false, isbig = false;
            if (v < n) {
#pragma unroll
                for (int i = 0; i < W; ++i) active = active || ld<CO>(cur + v * W + i) != 0ull;
                if (active) isbig = off[v + 1] - off[v] >= big_deg;
            }
            small[k] = active && !isbig;
            cnt += small[k];
            const unsigned bm = __ballot_sync(0xffffffffu, isbig);
            if (bm) {
                const int leader = __ffs(bm) - 1;
                unsigned long long b0 = 0;
                if ((int)lane == leader) b0 = atomicAdd(slot_cur + M_BIG, (unsigned long long)__popc(bm));
                b0 = __shfl_sync(0xffffffffu, b0, leader);
                if (isbig) big[b0 + __popc(bm & lanemask_lt())] = (int32_t)v;
            }
        }
        int tot;
        const int excl = warp_exclusive_scan(cnt, &tot);
        if (lane == 31) wtot[w] = tot;
        __syncthreads();
        int before = 0, all = 0;
        for (int i = 0; i < kMsBlock / 32; ++i) {
            if (i < (int)w) before += wtot[i];
            all += wtot[i];
        }
        if (threadIdx.x == 0) base_s = all ? atomicAdd(slot_cur + M_LIST, (unsigned long long)all) : 0ull;
        __syncthreads();
        unsigned long long pos = base_s + before + excl;
#pragma unroll
        for (int k = 0; k < per; ++k)
            if (small[k]) list[pos++] = (int32_t)(v0 + k);
        __syncthreads();
    }
}

// OR the frontier words `cu` of u into neighbour v's next words. The OR's
// old value is not used (the GPU does not wait on it), and no load of v's
// seen words filters it first: one random read per edge cost more than the
// ORs it saved; the keep-unseen pass masks seen bits out afterwards.
template <int W>
__device__ __forceinline__ void ms_push(const unsigned long long (&cu)[W], int64_t v,
                                        unsigned long long *__restrict__ nxt) {
#pragma unroll
    for (int i = 0; i < W; ++i)
        if (cu[i]) atomicOr(nxt + v * W + i, cu[i]);
}

// Top-down layer on bit lanes over the compacted list.
//   W = 1: a warp takes 32 entries; rows shorter than 32 are walked by their
//     own lane, longer ones by the whole warp.
//   W > 1: a group of W lanes (lane i = lane word i) takes one entry, so a
//     pushed edge is one broadcast index load and at most one atomicOr per
//     lane (none for a zero frontier word); the
//     32 / W groups of a warp take consecutive entries, 4 edges in flight;
//     rows of 32 or more edges are walked by the whole warp, group g on
//     edges g, g + 32 / W, ...
template <int W, bool CO>
__device__ __forceinline__ void ms_td_phase(
    const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
    const int32_t *__restrict__ list, const unsigned long long *slot_cur,
    const unsigned long long *__restrict__ cur, unsigned long long *__restrict__ nxt) {
    const int64_t cnt = (int64_t)ld<CO>(slot_cur + M_LIST);
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if constexpr (W > 1) {
        constexpr int G = 32 / W;  // groups per warp
        const int gid = (int)(lane / W), wi = (int)(lane % W);
        for (int64_t base = gw * G; base < cnt; base += tw * G) {
            const int64_t e_i = base + gid;
            int64_t beg = 0, end = 0;
            unsigned long long cu = 0ull;
            if (e_i < cnt) {
                const int64_t u = ld<CO>(list + e_i);
                beg = off[u];
                end = off[u + 1];
                cu = CO ? __ldcg(cur + u * W + wi) : __ldg(cur + u * W + wi);
            }
            if (end - beg < 32) {
                for (int64_t e = beg; e < end; e += 4) {
                    int64_t v[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) v[t] = e + t < end ? (int64_t)__ldg(idx + e + t) : -1;
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (v[t] >= 0 && cu) atomicOr(nxt + v[t] * W + wi, cu);
                }
            }
            // rows of 32 or more: the whole warp, one row at a time
            unsigned wm = __ballot_sync(0xffffffffu, wi == 0 && end - beg >= 32);
            while (wm) {
                const int L = __ffs(wm) - 1;
                wm &= wm - 1;
                const int64_t lb = __shfl_sync(0xffffffffu, beg, L);
                const int64_t le = __shfl_sync(0xffffffffu, end, L);
                const unsigned long long cL = __shfl_sync(0xffffffffu, cu, L + wi);
                for (int64_t e0 = lb + gid; e0 < le; e0 += 4 * G) {
                    int64_t v[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const int64_t e = e0 + (int64_t)t * G;
                        v[t] = e < le ? (int64_t)__ldg(idx + e) : -1;
                    }
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (v[t] >= 0 && cL) atomicOr(nxt + v[t] * W + wi, cL);
                }
            }
        }
    } else {
        for (int64_t base = gw * 32; base < cnt; base += tw * 32) {
            const int64_t i = base + lane;
            int64_t u = 0, beg = 0, end = 0;
            unsigned long long cu[W];
#pragma unroll
            for (int j = 0; j < W; ++j) cu[j] = 0ull;
            if (i < cnt) {
                u = ld<CO>(list + i);
                beg = off[u];
                end = off[u + 1];
                load_lanes<W, CO>(cur + u * W, cu);
            }
            const bool wide = end - beg >= 32;
            if (!wide) {
                // 4 edges in flight per lane
                for (int64_t e = beg; e < end; e += 4) {
                    int64_t v[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) v[t] = e + t < end ? (int64_t)__ldg(idx + e + t) : -1;
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (v[t] >= 0) ms_push<W>(cu, v[t], nxt);
                }
            }
            unsigned wm = __ballot_sync(0xffffffffu, wide);
            while (wm) {
                const int L = __ffs(wm) - 1;
                wm &= wm - 1;
                const int64_t lb = __shfl_sync(0xffffffffu, beg, L);
                const int64_t le = __shfl_sync(0xffffffffu, end, L);
                unsigned long long cL[W];
#pragma unroll
                for (int j = 0; j < W; ++j) cL[j] = __shfl_sync(0xffffffffu, cu[j], L);
                for (int64_t e = lb + lane; e < le; e += 32) ms_push<W>(cL, __ldg(idx + e), nxt);
            }
        }
    }
}

// The grid-spread list: batches of kMsBigBatch vertices, degree prefix in
// shared memory, grid-stride over the batch's edges.
template <int W, bool CO>
__device__ __forceinline__ void ms_td_big_phase(
    const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
    const int32_t *__restrict__ big, const unsigned long long *slot_cur,
    const unsigned long long *__restrict__ cur, unsigned long long *__restrict__ nxt) {
    __shared__ long long pre[kMsBigBatch + 1];
    __shared__ long long beg_s[kMsBigBatch];
    __shared__ int32_t u_s[kMsBigBatch];
    __shared__ long long wtot[kMsBlock / 32];
    const int64_t cnt = (int64_t)ld<CO>(slot_cur + M_BIG);
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tt = (int64_t)gridDim.x * blockDim.x;
    constexpr int per = kMsBigBatch / kMsBlock;
    for (int64_t b0 = 0; b0 < cnt; b0 += kMsBigBatch) {
        const int nb = (int)(cnt - b0 < kMsBigBatch ? cnt - b0 : kMsBigBatch);
        long long dsum = 0, dloc[per];
#pragma unroll
        for (int k = 0; k < per; ++k) {
            const int t = threadIdx.x * per + k;
            long long d = 0;
            if (t < nb) {
                const int32_t u = ld<CO>(big + b0 + t);
                u_s[t] = u;
                beg_s[t] = off[u];
                d = off[u + 1] - beg_s[t];
            }
            dloc[k] = d;
            dsum += d;
        }
        long long x = dsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) wtot[w] = x;
        __syncthreads();
        long long run = x - dsum;
        for (unsigned i = 0; i < w; ++i) run += wtot[i];
#pragma unroll
        for (int k = 0; k < per; ++k) {
            pre[threadIdx.x * per + k] = run;
            run += dloc[k];
        }
        if (threadIdx.x == kMsBlock - 1) pre[kMsBigBatch] = run;
        __syncthreads();
        const long long total = pre[kMsBigBatch];
        // one thread per edge with all W words: the owner search is shared
        // by the words (a group of W threads per edge measured slower here)
        for (long long g = gt; g < total; g += tt) {
            int lo = 0, hi = nb;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (pre[mid] <= g) lo = mid;
                else hi = mid;
            }
            unsigned long long cu[W];
            load_lanes<W, CO>(cur + (int64_t)u_s[lo] * W, cu);
            ms_push<W>(cu, __ldg(idx + beg_s[lo] + (g - pre[lo])), nxt);
        }
        __syncthreads();
    }
}

// After a top-down layer: keep the bits of nxt not yet seen (they become the
// next frontier), update seen and count; every vertex of degree >= 1 is
// checked for live roots it still lacks.
template <int W, bool CO>
__device__ __forceinline__ void ms_finalize_phase(
    const int64_t *__restrict__ off, const uint32_t *__restrict__ base_vis, int64_t n,
    Lanes<W> act, unsigned long long *__restrict__ seen, unsigned long long *__restrict__ nxt,
    int64_t td_edges, unsigned long long *slot_next, int64_t *zero_slot,
    unsigned long long *live_next, unsigned long long *live_zero) {
    if (blockIdx.x == 0 && threadIdx.x < 8) {
        zero_slot[threadIdx.x] = 0;
        live_zero[threadIdx.x] = 0ull;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t c[6] = {0, 0, 0, 0, 0, 0};
    unsigned long long nb[W];
#pragma unroll
    for (int i = 0; i < W; ++i) nb[i] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) c[5] = td_edges;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        if ((base_vis[v >> 5] >> (v & 31)) & 1u) continue;  // degree 0
        unsigned long long x[W], s[W], nw[W];
        load_lanes<W, CO>(nxt + v * W, x);
        load_lanes<W, CO>(seen + v * W, s);
        bool any = false;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            nw[i] = x[i] & ~s[i] & act.w[i];
            any = any || x[i] != 0ull;
        }
        if (any) {
#pragma unroll
            for (int i = 0; i < W; ++i) nxt[v * W + i] = nw[i];
        }
        ms_commit<W>(v, off[v + 1] - off[v], s, nw, act, seen, c, nb);
    }
    block_finish<W>(c, nb, slot_next, live_next);
}

// Per-byte x - 1 of eight bytes in [0, 128] (0 -> 0xFF), without borrows
// between bytes.
__device__ __forceinline__ unsigned long long bytes_dec(unsigned long long x) {
    constexpr unsigned long long H = 0x8080808080808080ull, L = 0x0101010101010101ull;
    return ((x | H) - L) ^ ((x ^ ~L) & H);
}

// Level rows from the frontier slots of layers [j_lo, j_hi), one tile of
// C = kMsBlock / W consecutive vertices (columns) per block and step: thread
// t owns lane word i = t % W of vertex v0 + t / W, so each layer's frontier
// words of the tile are one contiguous load by the block.
//   full = 1: every row r < k of the tile's columns is written, -1 where none
//     of the layers holds the bit. A thread builds the 64 levels of its
//     (vertex, word) as bit planes: plane p ORs the frontier words of the
//     layers j whose j + 1 has bit p set, so bit b of plane p is bit p of
//     level + 1 of root 64i + b. Per group of 8 roots, the 8 plane bytes are
//     gathered by byte permutes into an 8 x 8 bit matrix whose transpose
//     holds the 8 level + 1 bytes (then minus 1: 0 -> -1). The bytes go to a
//     shared tile of 64W rows x C bytes, the rows of word i rotated by
//     i * C / 8 bytes so that a warp's byte stores hit distinct banks; then
//     each warp stores whole rows, 4 or 8 bytes per lane, 128 or 256 bytes
//     per store instruction (whole sectors).
//   full = 0: only the reached pairs are written (layers after an earlier
//     full pass).
// vec: n and the level buffer allow 8-byte aligned row stores.
template <int W, bool CO>
__device__ __forceinline__ void ms_levels_phase(const unsigned long long *__restrict__ fr,
                                                int64_t slot_words, int lcap, int j_lo, int j_hi,
                                                int64_t n, int k, int8_t *__restrict__ levels,
                                                int full, int vec) {
    constexpr int C = kMsBlock / W;  // columns of a tile
    constexpr int R = 64 * W;        // rows of a tile (roots)
    constexpr int CP = C + 8;        // padded row stride in bytes
    constexpr int SW = C / 8;        // rotation of word i's rows: i * SW bytes
    __shared__ __align__(16) uint8_t tile[R * CP];
    const int i = (int)(threadIdx.x % W), vl = (int)(threadIdx.x / W);
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const int rows = k < R ? k : R;
    const int64_t ntiles = (n + C - 1) / C;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t v0 = tl * C, v = v0 + vl;
        const bool inb = v < n && i * 64 < k;
        if (full) {
            unsigned long long P[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) P[q] = 0ull;
            int sj = j_lo % lcap;
            for (int j = j_lo; j < j_hi; ++j) {
                const unsigned long long m =
                    inb ? ld<CO>(fr + (int64_t)sj * slot_words + v * W + i) : 0ull;
                const unsigned jj = (unsigned)(j + 1);  // the same in every thread
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if ((jj >> q) & 1u) P[q] |= m;
                sj = sj + 1 == lcap ? 0 : sj + 1;
            }
            uint8_t *col = tile + (i * 64) * CP + ((vl + i * SW) % C);
#pragma unroll
            for (int g = 0; g < 8; ++g) {
                // byte q of x = byte g of plane q (row q of an 8 x 8 bit matrix)
                const unsigned sel = (unsigned)(g & 3) | ((4u + (unsigned)(g & 3)) << 4);
                unsigned w[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) w[q] = (unsigned)(P[q] >> (32 * (g >> 2)));
                const unsigned lo = __byte_perm(__byte_perm(w[0], w[1], sel),
                                                __byte_perm(w[2], w[3], sel), 0x5410);
                const unsigned hi = __byte_perm(__byte_perm(w[4], w[5], sel),
                                                __byte_perm(w[6], w[7], sel), 0x5410);
                unsigned long long x = ((unsigned long long)hi << 32) | lo;
                // transpose: bit t of byte q -> bit q of byte t
                unsigned long long t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
                x = x ^ t ^ (t << 7);
                t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
                x = x ^ t ^ (t << 14);
                t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
                x = x ^ t ^ (t << 28);
                x = bytes_dec(x);
#pragma unroll
                for (int b = 0; b < 8; ++b) col[(8 * g + b) * CP] = (uint8_t)(x >> (8 * b));
            }
            __syncthreads();
            const bool whole = vec && v0 + C <= n;
            if (whole) {
                // each lane stores BL bytes; a store instruction covers RS rows
                constexpr int BL = C >= 256 ? 8 : 4;
                constexpr int LPR = C / BL;       // lanes per row
                constexpr int RS = 32 / LPR;      // rows per store instruction
                const int rr = (int)lane / LPR, cb = ((int)lane % LPR) * BL;
                for (int r0 = (int)warp * RS; r0 < rows; r0 += (kMsBlock / 32) * RS) {
                    const int r = r0 + rr;
                    if (r >= rows) continue;
                    // columns [cb, cb + BL) sit at (cb + rotation) % C, a
                    // multiple of BL: the BL bytes stay together
                    const uint8_t *src = tile + r * CP + ((cb + (r / 64) * SW) % C);
                    int8_t *dst = levels + (int64_t)r * n + v0 + cb;
                    if constexpr (BL == 8)
                        *reinterpret_cast<unsigned long long *>(dst) =
                            *reinterpret_cast<const unsigned long long *>(src);
                    else
                        *reinterpret_cast<uint32_t *>(dst) = *reinterpret_cast<const uint32_t *>(src);
                }
            } else {
                for (int r = (int)warp; r < rows; r += kMsBlock / 32) {
                    int8_t *dst = levels + (int64_t)r * n + v0;
                    const uint8_t *src = tile + r * CP;
                    const int rot = (r / 64) * SW;
                    for (int c = (int)lane; c < C; c += 32)
                        if (v0 + c < n) dst[c] = (int8_t)src[(c + rot) % C];
                }
            }
            __syncthreads();
        } else if (inb) {
            for (int j = j_lo; j < j_hi; ++j) {
                unsigned long long m = ld<CO>(fr + (int64_t)(j % lcap) * slot_words + v * W + i);
                while (m) {
                    const int b = __ffsll((long long)m) - 1;
                    m &= m - 1;
                    if (i * 64 + b < k) levels[(int64_t)(i * 64 + b) * n + v] = (int8_t)j;
                }
            }
        }
    }
}

// Kernels for the host-driven loop: one phase each.
template <int W>
__global__ void __launch_bounds__(kMsBlock) ms_bu_kernel(
    const int64_t *off, const int32_t *idx, const uint32_t *base_vis, int64_t n, Lanes<W> act,
    unsigned long long *seen, const unsigned long long *cur, unsigned long long *nxt, int probe,
    unsigned long long *slot_next, int64_t *zero_slot, unsigned long long *live_next,
    unsigned long long *live_zero) {
    ms_bu_phase<W, false>(off, idx, base_vis, n, act, seen, cur, nxt, probe, slot_next, zero_slot,
                          live_next, live_zero);
}

template <int W>
__global__ void __launch_bounds__(kMsBlock) ms_compact_kernel(
    const unsigned long long *cur, int64_t n, const int64_t *off, int64_t big_deg, int32_t *list,
    int32_t *big, unsigned long long *slot_cur) {
    ms_compact_phase<W, false>(cur, n, off, big_deg, list, big, slot_cur);
}

template <int W>
__global__ void __launch_bounds__(kMsBlock) ms_td_kernel(
    const int64_t *off, const int32_t *idx, const int32_t *list, const unsigned long long *slot_cur,
    const unsigned long long *cur, unsigned long long *nxt) {
    ms_td_phase<W, false>(off, idx, list, slot_cur, cur, nxt);
}

template <int W>
__global__ void __launch_bounds__(kMsBlock) ms_td_big_kernel(
    const int64_t *off, const int32_t *idx, const int32_t *big, const unsigned long long *slot_cur,
    const unsigned long long *cur, unsigned long long *nxt) {
    ms_td_big_phase<W, false>(off, idx, big, slot_cur, cur, nxt);
}

template <int W>
__global__ void __launch_bounds__(kMsBlock) ms_finalize_kernel(
    const int64_t *off, const uint32_t *base_vis, int64_t n, Lanes<W> act,
    unsigned long long *seen, unsigned long long *nxt, int64_t td_edges,
    unsigned long long *slot_next, int64_t *zero_slot, unsigned long long *live_next,
    unsigned long long *live_zero) {
    ms_finalize_phase<W, false>(off, base_vis, n, act, seen, nxt, td_edges, slot_next, zero_slot,
                                live_next, live_zero);
}

template <int W>
__global__ void __launch_bounds__(kMsBlock) ms_levels_kernel(
    const unsigned long long *fr, int64_t slot_words, int lcap, int j_lo, int j_hi, int64_t n,
    int k, int8_t *levels, int full, int vec) {
    ms_levels_phase<W, false>(fr, slot_words, lcap, j_lo, j_hi, n, k, levels, full, vec);
}

struct MsPersist {
    const int64_t *off;
    const int32_t *idx;
    const uint32_t *base_vis;
    int64_t n, nnz;
    unsigned long long *seen, *fr, *live;
    int64_t slot_words;
    int lcap, k, vec;
    int8_t *levels;
    int32_t *list, *big;
    int64_t *trace;   // ring of kMsRingP slots; slot 0 written by ms_roots_kernel
    int64_t *layers;  // [128][8] per-layer record
    int32_t *result;  // [0] layers, [1] status
    unsigned *bar;    // barrier count, generation
    int32_t *err;
    double alpha, beta;
    int probe;
    int64_t big_deg;
    unsigned long long timeout_ns;
};

constexpr int kMsRingP = 64;
constexpr int kMsFieldsP = 8;

// The whole batched traversal in one cooperative launch: every block runs
// the same layer loop and takes the same direction decision from the layer
// counters and live mask, which grid barriers make visible between phases.
// Bottom-up layers are one phase; top-down layers are compaction (+ clearing
// the next slot), push, and the dense keep-unseen pass. The level rows are
// written by a last phase (and by a flush phase when the slot ring is full).
template <int W>
__global__ void __launch_bounds__(kMsBlock) ms_persistent_kernel(MsPersist p) {
    const unsigned expected = gridDim.x;
    int64_t e_u = __ldcg(p.trace + M_LACKDEG);
    int64_t v_u = __ldcg(p.trace + M_LACKN);
    int cur_bu = 0, status = BFS_OK, d = 0, j_lo = 0, flushed = 0;
    for (;; ++d) {
        int64_t *sc = p.trace + (d % kMsRingP) * kMsFieldsP;
        int64_t *sn = p.trace + ((d + 1) % kMsRingP) * kMsFieldsP;
        int64_t *sz = p.trace + ((d + 2) % kMsRingP) * kMsFieldsP;
        const int64_t v_f = __ldcg(sc + M_NV), e_f = __ldcg(sc + M_MF);
        if (d > 0 && d - 1 < kPctlLayers && blockIdx.x == 0 && threadIdx.x == 0)
            p.layers[(int64_t)(d - 1) * 8 + 6] = __ldcg(sc + M_EXAM);  // the last layer's edges
        if (v_f == 0) break;
        if (d + 1 > 127) {
            status = BFS_ERR_DEPTH;
            break;
        }
        if (d + 1 - j_lo >= p.lcap) {  // the next slot still holds an unwritten layer
            ms_levels_phase<W, true>(p.fr, p.slot_words, p.lcap, j_lo, d + 1, p.n, p.k, p.levels,
                                     !flushed, p.vec);
            flushed = 1;
            j_lo = d + 1;
            if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
                status = BFS_ERR_TIMEOUT;
                break;
            }
        }
        if (!cur_bu) cur_bu = ((double)e_f > (double)e_u / p.alpha) ? 1 : 0;
        else cur_bu = ((double)v_f < (double)p.n / p.beta) ? 0 : 1;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            int64_t *rec = p.layers + (int64_t)d * 8;
            rec[0] = cur_bu;
            rec[1] = v_f;
            rec[2] = e_f;
            rec[3] = __ldcg(sc + M_PAIRS);
            rec[4] = v_u;
            rec[5] = e_u;
        }
        const Lanes<W> act = load_live<W>(p.live + (d % 3) * 8);
        unsigned long long *live_next = p.live + ((d + 1) % 3) * 8;
        unsigned long long *live_zero = p.live + ((d + 2) % 3) * 8;
        unsigned long long *cur = p.fr + (int64_t)(d % p.lcap) * p.slot_words;
        unsigned long long *nxt = p.fr + (int64_t)((d + 1) % p.lcap) * p.slot_words;
        if (cur_bu) {
            ms_bu_phase<W, true>(p.off, p.idx, p.base_vis, p.n, act, p.seen, cur, nxt, p.probe,
                                 (unsigned long long *)sn, sz, live_next, live_zero);
        } else {
            int64_t bd = e_f / ((int64_t)gridDim.x * (kMsBlock / 32) * (W > 1 ? 32 / W : 1));
            bd = bd < 32 ? 32 : (bd > p.big_deg ? p.big_deg : bd);
            ms_compact_phase<W, true>(cur, p.n, p.off, bd, p.list, p.big,
                                      (unsigned long long *)sc);
            const int64_t stride = (int64_t)gridDim.x * blockDim.x;
            for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.slot_words;
                 i += stride)
                nxt[i] = 0ull;
            if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
                status = BFS_ERR_TIMEOUT;
                break;
            }
            ms_td_phase<W, true>(p.off, p.idx, p.list, (const unsigned long long *)sc, cur, nxt);
            ms_td_big_phase<W, true>(p.off, p.idx, p.big, (const unsigned long long *)sc, cur, nxt);
            if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
                status = BFS_ERR_TIMEOUT;
                break;
            }
            ms_finalize_phase<W, true>(p.off, p.base_vis, p.n, act, p.seen, nxt, e_f,
                                       (unsigned long long *)sn, sz, live_next, live_zero);
        }
        if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
            status = BFS_ERR_TIMEOUT;
            break;
        }
        v_u = __ldcg(sn + M_LACKN);
        e_u = __ldcg(sn + M_LACKDEG);
    }
    if (status != BFS_ERR_TIMEOUT)  // levels of the layers still in the ring
        ms_levels_phase<W, true>(p.fr, p.slot_words, p.lcap, j_lo, d + 1, p.n, p.k, p.levels,
                                 !flushed, p.vec);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.result[0] = d;
        p.result[1] = status;
    }
}

// One barrier that waits for `missing` more blocks than the grid has: the
// wait runs out and the kernel reports it instead of hanging.
__global__ void barrier_probe_kernel(unsigned *bar, int32_t *err, unsigned missing,
                                     unsigned long long timeout_ns, int32_t *ok) {
    const bool r = grid_barrier(bar, err, gridDim.x + missing, timeout_ns);
    if (threadIdx.x == 0 && !r) atomicExch(ok, 0);
}

}  // namespace
}  // namespace gbfs

namespace gbfs {
namespace {

constexpr int kMsRing = 64;
constexpr int kMsFields = 8;

bool batch_cfg_ok(const bfs_batch_config &c) {
    return c.alpha > 0 && c.beta > 0 && c.lane_probe >= 0 && c.lane_probe <= 4096 &&
           c.big_degree >= 32 && (c.use_graph == 0 || c.use_graph == 1) &&
           (c.layer_slots == 0 || (c.layer_slots >= 2 && c.layer_slots <= kMaxSlots));
}

// Bitsets for W lane words: seen and the frontier slot ring. The ring gets
// cfg.layer_slots slots, or (0) as many as a quarter of the free device
// memory holds, 4 to 16.
bfs_status ensure_ms(bfs_graph *g, int W) {
    if (!g->ms) {
        g->ms = new MsState();
        bfs_batch_config_default(&g->ms->cfg);
        g->ms->n = g->n;
    }
    MsState *m = g->ms;
    if (!m->list) {
        GB_CK(dev_malloc(&m->list, (size_t)g->n * 4));
        GB_CK(dev_malloc(&m->big, (size_t)g->n * 4));
        GB_CK(dev_malloc(&m->roots, kMaxRoots * 4));
        GB_CK(dev_malloc(&m->trace, (size_t)kMsRing * kMsFields * 8));
        GB_CK(dev_malloc(&m->live, 3 * 8 * 8));
        GB_CK(host_malloc(&m->h_slot, 16 * 8));
        GB_CK(host_malloc((void **)&m->h_pub, 17 * 8, cudaHostAllocMapped));
        GB_CK(cudaHostGetDevicePointer((void **)&m->d_pub, m->h_pub, 0));
        m->h_pub[16] = 0;
    }
    if (W == 0) return BFS_OK;
    const int want = m->cfg.layer_slots;
    if (m->W < W || (want > 0 && want != m->lcap)) {
        cudaFree(m->seen);
        cudaFree(m->fr);
        m->seen = m->fr = nullptr;
        m->W = 0;
        m->lcap = 0;
        const size_t slot = (size_t)g->n * W * 8;
        int lcap = want;
        if (lcap == 0) {
            size_t fb = 0, tb = 0;
            GB_CK(cudaMemGetInfo(&fb, &tb));
            lcap = (int)std::max<size_t>(4, std::min<size_t>(kMaxSlots, fb / 4 / slot));
        }
        GB_CK(dev_malloc(&m->seen, slot));
        GB_CK(dev_malloc(&m->fr, slot * lcap));
        m->W = W;
        m->lcap = lcap;
    }
    return BFS_OK;
}

// Copies a trace slot and a live mask into the mapped host block, then,
// after a system fence, the sequence number the host waits for.
__global__ void ms_publish_kernel(const int64_t *__restrict__ slot,
                                  const unsigned long long *__restrict__ live, int64_t *pub,
                                  int64_t seq) {
    if (threadIdx.x == 0) {
        volatile int64_t *vp = pub;
        for (int i = 0; i < 8; ++i) vp[i] = slot[i];
        for (int i = 0; i < 8; ++i) vp[8 + i] = (int64_t)live[i];
        __threadfence_system();
        vp[16] = seq;
    }
}

// Publishes a layer's counters and live mask and spins on the sequence
// number in mapped memory (instead of a copy and a stream synchronisation);
// after 5 s the stream is synchronised, which returns a failed kernel's
// error. The values land in m->h_slot[0..16).
bfs_status ms_publish_and_wait(MsState *m, const int64_t *slot, const unsigned long long *live,
                               cudaStream_t st) {
    const int64_t seq = ++m->pub_seq;
    ms_publish_kernel<<<1, 32, 0, st>>>(slot, live, m->d_pub, seq);
    count_launch();
    GB_CK(cudaGetLastError());
    volatile int64_t *vp = m->h_pub;
    const auto t0 = std::chrono::steady_clock::now();
    for (long spins = 0; vp[16] != seq; ++spins) {
        if ((spins & 1023) == 1023) {
            if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(5)) {
                GB_CK(cudaStreamSynchronize(st));
                if (vp[16] != seq) {
                    set_error("bfs_run_batch: the layer counters never arrived");
                    return BFS_ERR_CUDA;
                }
                break;
            }
            if (spins > (1 << 16)) std::this_thread::yield();
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    for (int i = 0; i < 16; ++i) m->h_slot[i] = vp[i];
    return BFS_OK;
}

// Slots of the ring when it runs W lane words (a ring sized for wider words
// holds more narrower slots).
int ring_slots(const MsState *m, int W) {
    return std::min(kMaxSlots, m->lcap * (m->W / W));
}

template <int W>
Lanes<W> active_lanes(int k) {
    Lanes<W> a;
    for (int i = 0; i < W; ++i) {
        const int bits = std::max(0, std::min(64, k - 64 * i));
        a.w[i] = bits == 64 ? ~0ull : ((1ull << bits) - 1ull);
    }
    return a;
}

template <int W>
bfs_status run_batch_w(bfs_graph *g, const int32_t *roots, int k, int8_t *levels, cudaStream_t st) {
    MsState *m = g->ms;
    const bfs_batch_config &cfg = m->cfg;
    const int64_t n = g->n;
    Lanes<W> act = active_lanes<W>(k);
    unsigned long long *seen = m->seen;
    const int64_t slot_words = n * W;
    const int lcap = ring_slots(m, W);
    const bool timing = cfg.timing != 0;
    auto event = [&](size_t i) -> cudaEvent_t {
        while (m->events.size() <= i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            m->events.push_back(e);
        }
        return m->events[i];
    };
    int bu_occ = 1, td_occ = 1, lv_occ = 1;
    GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu_occ, ms_bu_kernel<W>, kMsBlock, 0));
    GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&td_occ, ms_td_kernel<W>, kMsBlock, 0));
    GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&lv_occ, ms_levels_kernel<W>, kMsBlock, 0));
    const int64_t ntiles = (n + kMsBlock / W - 1) / (kMsBlock / W);
    const int vec = (n % 8 == 0 && (uintptr_t)levels % 8 == 0) ? 1 : 0;
    auto write_levels = [&](int j_lo, int j_hi, int full) -> bfs_status {
        GB_LAUNCH(ms_levels_kernel<W>, grid_cap(ntiles, 1, lv_occ), kMsBlock, 0, st, m->fr,
                  slot_words, lcap, j_lo, j_hi, n, k, levels, full, vec);
        return BFS_OK;
    };
    GB_LAUNCH(ms_fill_kernel, grid_cap(n * W, kMsBlock, 8), kMsBlock, 0, st, seen, m->fr, n * W);
    GB_CK(cudaMemsetAsync(m->trace, 0, (size_t)kMsRing * kMsFields * 8, st));
    GB_LAUNCH(ms_roots_kernel<W>, 1, kMaxRoots, 0, st, roots, k, n, n - g->deg0, g->nnz, g->off,
              act, seen, m->fr, m->live, m->trace);
    {
        const bfs_status ps = ms_publish_and_wait(m, m->trace, m->live, st);
        if (ps != BFS_OK) return ps;
    }
    int64_t v_f = m->h_slot[M_NV], e_f = m->h_slot[M_MF], pairs = k;
    int64_t v_u = m->h_slot[M_LACKN], e_u = m->h_slot[M_LACKDEG];
    m->last.clear();
    m->last_pairs = k;
    int cur_bu = 0, j_lo = 0, flushed = 0, d = 0;
    const int64_t nwords = (n + 31) / 32;
    const int bu_grid = grid_cap(nwords, kMsBlock / 32, bu_occ);
    const int64_t td_warps = (int64_t)sm_count() * td_occ * (kMsBlock / 32);
    for (d = 0; v_f > 0; ++d) {
        if (d + 1 > 127) {
            bfs_status s = write_levels(j_lo, d + 1, !flushed);
            if (s == BFS_OK) GB_CK(cudaStreamSynchronize(st));
            set_error("bfs_run_batch: a level above 127 does not fit in int8");
            return s == BFS_OK ? BFS_ERR_DEPTH : s;
        }
        if (d + 1 - j_lo >= lcap) {  // the next slot still holds an unwritten layer
            bfs_status s = write_levels(j_lo, d + 1, !flushed);
            if (s != BFS_OK) return s;
            flushed = 1;
            j_lo = d + 1;
        }
        if (!cur_bu) cur_bu = ((double)e_f > (double)e_u / cfg.alpha) ? 1 : 0;
        else cur_bu = ((double)v_f < (double)n / cfg.beta) ? 0 : 1;
        bfs_batch_layer_stats ls;
        memset(&ls, 0, sizeof ls);
        ls.direction = cur_bu;
        ls.v_f = v_f;
        ls.e_f = e_f;
        ls.pairs = pairs;
        ls.v_u = v_u;
        ls.e_u = e_u;
        int64_t *slot_cur = m->trace + (d % kMsRing) * kMsFields;
        int64_t *slot_next = m->trace + ((d + 1) % kMsRing) * kMsFields;
        int64_t *slot_zero = m->trace + ((d + 2) % kMsRing) * kMsFields;
        unsigned long long *live_next = m->live + ((d + 1) % 3) * 8;
        unsigned long long *live_zero = m->live + ((d + 2) % 3) * 8;
        unsigned long long *cur = m->fr + (int64_t)(d % lcap) * slot_words;
        unsigned long long *nxt = m->fr + (int64_t)((d + 1) % lcap) * slot_words;
        if (timing) GB_CK(cudaEventRecord(event(2 * d), st));
        if (cur_bu) {
            GB_LAUNCH(ms_bu_kernel<W>, bu_grid, kMsBlock, 0, st, g->off, g->idx, g->base_vis, n,
                      act, seen, cur, nxt, cfg.lane_probe, (unsigned long long *)slot_next,
                      slot_zero, live_next, live_zero);
        } else {
            // grid-spread threshold: the frontier's edges per resident row
            // walker (a warp for W = 1, a group of W lanes otherwise),
            // clamped to [32, big_degree]
            const int64_t big_deg = std::max<int64_t>(
                32, std::min<int64_t>(cfg.big_degree, e_f / (td_warps * (W > 1 ? 32 / W : 1))));
            GB_LAUNCH(ms_compact_kernel<W>, grid_cap(n, kMsBlock * 4, 8), kMsBlock, 0, st, cur, n,
                      g->off, big_deg, m->list, m->big, (unsigned long long *)slot_cur);
            GB_CK(cudaMemsetAsync(nxt, 0, (size_t)slot_words * 8, st));
            GB_LAUNCH(ms_td_kernel<W>, grid_cap(v_f, kMsBlock, td_occ), kMsBlock, 0, st, g->off,
                      g->idx, m->list, (const unsigned long long *)slot_cur, cur, nxt);
            if (e_f >= big_deg)
                GB_LAUNCH(ms_td_big_kernel<W>,
                          (int)std::max<int64_t>(1, std::min<int64_t>(e_f / 2048 + 1,
                                                                      (int64_t)sm_count() * 4)),
                          kMsBlock, 0, st, g->off, g->idx, m->big,
                          (const unsigned long long *)slot_cur, cur, nxt);
            GB_LAUNCH(ms_finalize_kernel<W>, grid_cap(n, kMsBlock, 8), kMsBlock, 0, st, g->off,
                      g->base_vis, n, act, seen, nxt, e_f, (unsigned long long *)slot_next,
                      slot_zero, live_next, live_zero);
        }
        if (timing) GB_CK(cudaEventRecord(event(2 * d + 1), st));
        {
            const bfs_status ps = ms_publish_and_wait(m, slot_next, live_next, st);
            if (ps != BFS_OK) return ps;
        }
        ls.examined = m->h_slot[M_EXAM];
        m->last.push_back(ls);
        v_f = m->h_slot[M_NV];
        e_f = m->h_slot[M_MF];
        pairs = m->h_slot[M_PAIRS];
        m->last_pairs += pairs;
        v_u = m->h_slot[M_LACKN];
        e_u = m->h_slot[M_LACKDEG];
        for (int i = 0; i < W; ++i) act.w[i] = (unsigned long long)m->h_slot[8 + i];
    }
    bfs_status s = write_levels(j_lo, d + 1, !flushed);
    if (s != BFS_OK) return s;
    GB_CK(cudaStreamSynchronize(st));
    if (timing)
        for (size_t i = 0; i < m->last.size(); ++i)
            cudaEventElapsedTime(&m->last[i].ms, m->events[2 * i], m->events[2 * i + 1]);
    return BFS_OK;
}

constexpr size_t kPctlBytes = kPctlLayers * 8 * 8 + 64;  // records, result, barrier, err

// The same traversal as run_batch_w, as one CUDA graph: clearing, roots and
// the persistent kernel (a cooperative node). The graph is captured once per
// (W, k, output buffer, bitset buffers, configuration) and replayed.
template <int W>
bfs_status run_batch_graph(bfs_graph *g, const int32_t *roots, int k, int8_t *levels,
                           cudaStream_t st) {
    MsState *m = g->ms;
    const int64_t n = g->n;
    if (!m->pctl) {
        GB_CK(dev_malloc(&m->pctl, kPctlBytes));
        GB_CK(host_malloc(&m->h_pctl, kPctlBytes));
    }
    const bool stale = !m->exec || m->g_W != W || m->g_k != k || m->g_levels != levels ||
                       m->g_seen != m->seen || memcmp(&m->g_cfg, &m->cfg, sizeof m->cfg) != 0;
    if (stale) {
        if (m->exec) cudaGraphExecDestroy(m->exec);
        if (m->graph) cudaGraphDestroy(m->graph);
        m->exec = nullptr;
        m->graph = nullptr;
        int occ = 0;
        GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ms_persistent_kernel<W>,
                                                            kMsBlock, 0));
        if (occ < 1) {
            set_error("bfs_run_batch: the persistent kernel does not fit on an SM");
            return BFS_ERR_CUDA;
        }
        const Lanes<W> act = active_lanes<W>(k);
        MsPersist p;
        p.off = g->off;
        p.idx = g->idx;
        p.base_vis = g->base_vis;
        p.n = n;
        p.nnz = g->nnz;
        p.seen = m->seen;
        p.fr = m->fr;
        p.live = m->live;
        p.slot_words = n * W;
        p.lcap = ring_slots(m, W);
        p.k = k;
        p.vec = (n % 8 == 0 && (uintptr_t)levels % 8 == 0) ? 1 : 0;
        p.levels = levels;
        p.list = m->list;
        p.big = m->big;
        p.trace = m->trace;
        p.layers = m->pctl;
        p.result = (int32_t *)(m->pctl + kPctlLayers * 8);
        p.bar = (unsigned *)(p.result + 2);
        p.err = (int32_t *)(p.bar + 2);
        p.alpha = m->cfg.alpha;
        p.beta = m->cfg.beta;
        p.probe = m->cfg.lane_probe;
        p.big_deg = m->cfg.big_degree;
        p.timeout_ns = 2000000000ull;  // 2 s per barrier wait
        // Captured on a private stream (capture cannot start on the legacy
        // default stream); the instantiated graph is launched on `st`.
        if (!m->cap) GB_CK(cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking));
        cudaStream_t cs = m->cap;
        GB_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        ms_fill_kernel<<<grid_cap(n * W, kMsBlock, 8), kMsBlock, 0, cs>>>(m->seen, m->fr, n * W);
        cudaMemsetAsync(m->trace, 0, (size_t)kMsRing * kMsFields * 8, cs);
        ms_roots_kernel<W><<<1, kMaxRoots, 0, cs>>>(roots, k, n, n - g->deg0, g->nnz, g->off, act,
                                                    m->seen, m->fr, m->live, m->trace);
        cudaMemsetAsync(p.result, 0, 64, cs);
        cudaLaunchConfig_t lc;
        memset(&lc, 0, sizeof lc);
        lc.gridDim = dim3(occ * sm_count());
        lc.blockDim = dim3(kMsBlock);
        lc.stream = cs;
        cudaLaunchAttribute at;
        at.id = cudaLaunchAttributeCooperative;
        at.val.cooperative = 1;
        lc.attrs = &at;
        lc.numAttrs = 1;
        cudaError_t le = cudaLaunchKernelEx(&lc, ms_persistent_kernel<W>, p);
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return cuda_status(le != cudaSuccess ? le : ce, "capture of the batched traversal",
                               __FILE__, __LINE__);
        }
        m->graph = graph;
        GB_CK(cudaGraphInstantiate(&m->exec, graph, 0));
        m->g_W = W;
        m->g_k = k;
        m->g_levels = levels;
        m->g_seen = m->seen;
        m->g_cfg = m->cfg;
    }
    GB_CK(cudaGraphLaunch(m->exec, st));
    count_launch(3);
    GB_CK(cudaMemcpyAsync(m->h_pctl, m->pctl, kPctlBytes, cudaMemcpyDeviceToHost, st));
    GB_CK(cudaStreamSynchronize(st));
    const int32_t *res = (const int32_t *)(m->h_pctl + kPctlLayers * 8);
    const int L = std::min(res[0], kPctlLayers);
    m->last.clear();
    m->last_pairs = 0;
    for (int d = 0; d < L; ++d) {
        const int64_t *rec = m->h_pctl + (int64_t)d * 8;
        bfs_batch_layer_stats ls;
        memset(&ls, 0, sizeof ls);
        ls.direction = (int32_t)rec[0];
        ls.v_f = rec[1];
        ls.e_f = rec[2];
        ls.pairs = rec[3];
        ls.v_u = rec[4];
        ls.e_u = rec[5];
        ls.examined = rec[6];
        m->last.push_back(ls);
        m->last_pairs += ls.pairs;
    }
    if (res[1] == BFS_ERR_DEPTH) {
        set_error("bfs_run_batch: a level above 127 does not fit in int8");
        return BFS_ERR_DEPTH;
    }
    if (res[1] != BFS_OK) {
        set_error("bfs_run_batch: a grid barrier wait of the device loop ran out");
        return (bfs_status)res[1];
    }
    return BFS_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace gbfs
using namespace gbfs;

extern "C" BFS_API void bfs_batch_config_default(bfs_batch_config *c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    // the autotuner's choice on R-MAT scale 22, k = 64..512: top-down until
    // the frontier is most of the graph, then bottom-up to the end
    c->alpha = 1.0;
    c->beta = 1e9;
    c->lane_probe = 4;
    c->big_degree = 4096;
    c->use_graph = 0;
    c->timing = 0;
}

extern "C" BFS_API bfs_status bfs_graph_set_batch_config(bfs_graph *g, const bfs_batch_config *cfg) {
    clear_error();
    if (!g) {
        set_error("bfs_graph_set_batch_config: null graph");
        return BFS_ERR_INVALID;
    }
    bfs_batch_config c;
    if (cfg) c = *cfg;
    else bfs_batch_config_default(&c);
    if (!batch_cfg_ok(c)) {
        set_error("bfs_graph_set_batch_config: invalid configuration");
        return BFS_ERR_INVALID;
    }
    bfs_status s = ensure_ms(g, 0);
    if (s != BFS_OK) return s;
    g->ms->cfg = c;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_graph_get_batch_config(const bfs_graph *g, bfs_batch_config *cfg) {
    clear_error();
    if (!g || !cfg) {
        set_error("bfs_graph_get_batch_config: null argument");
        return BFS_ERR_INVALID;
    }
    if (g->ms) *cfg = g->ms->cfg;
    else bfs_batch_config_default(cfg);
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_run_batch(bfs_graph *g, const int32_t *roots, int32_t k,
                                            int8_t *levels_out, void *stream) {
    clear_error();
    if (!g || !roots || !levels_out || k < 1 || k > kMaxRoots) {
        set_error("bfs_run_batch: need a graph, roots, levels_out and 1 <= k <= %d", kMaxRoots);
        return BFS_ERR_INVALID;
    }
    cudaStream_t st = as_stream(stream);
    const int W = k <= 64 ? 1 : k <= 128 ? 2 : k <= 256 ? 4 : 8;
    bfs_status s = ensure_ms(g, W);
    if (s != BFS_OK) return s;
    MsState *m = g->ms;
    // roots are validated on the host (copied there first if they are device memory)
    std::vector<int32_t> hr(k);
    if (is_device_ptr(roots)) {
        GB_CK(cudaMemcpyAsync(hr.data(), roots, (size_t)k * 4, cudaMemcpyDeviceToHost, st));
        GB_CK(cudaStreamSynchronize(st));
    } else {
        memcpy(hr.data(), roots, (size_t)k * 4);
    }
    for (int i = 0; i < k; ++i)
        if (hr[i] < 0 || hr[i] >= g->n) {
            set_error("bfs_run_batch: root %d = %d is outside [0, n)", i, hr[i]);
            return BFS_ERR_INVALID;
        }
    GB_CK(cudaMemcpyAsync(m->roots, hr.data(), (size_t)k * 4, cudaMemcpyHostToDevice, st));
    if (m->cfg.use_graph) {
        switch (W) {
            case 1: return run_batch_graph<1>(g, m->roots, k, levels_out, st);
            case 2: return run_batch_graph<2>(g, m->roots, k, levels_out, st);
            case 4: return run_batch_graph<4>(g, m->roots, k, levels_out, st);
            default: return run_batch_graph<8>(g, m->roots, k, levels_out, st);
        }
    }
    switch (W) {
        case 1: return run_batch_w<1>(g, m->roots, k, levels_out, st);
        case 2: return run_batch_w<2>(g, m->roots, k, levels_out, st);
        case 4: return run_batch_w<4>(g, m->roots, k, levels_out, st);
        default: return run_batch_w<8>(g, m->roots, k, levels_out, st);
    }
}

extern "C" BFS_API bfs_status bfs_last_batch_stats(const bfs_graph *g, bfs_batch_layer_stats *out,
                                                   int32_t cap, int32_t *layers,
                                                   int64_t *pairs_reached) {
    clear_error();
    if (!g || cap < 0 || (cap > 0 && !out)) {
        set_error("bfs_last_batch_stats: null graph or output");
        return BFS_ERR_INVALID;
    }
    const int32_t L = g->ms ? (int32_t)g->ms->last.size() : 0;
    for (int32_t i = 0; i < std::min(cap, L); ++i) out[i] = g->ms->last[i];
    if (layers) *layers = L;
    if (pairs_reached) *pairs_reached = g->ms ? g->ms->last_pairs : 0;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_batch_autotune(bfs_graph *g, const int32_t *roots, int32_t k,
                                                 int8_t *levels_scratch, bfs_batch_config *best,
                                                 void *stream) {
    clear_error();
    if (!g || !roots || !levels_scratch || k < 1 || k > kMaxRoots) {
        set_error("bfs_batch_autotune: need a graph, roots, scratch and 1 <= k <= %d", kMaxRoots);
        return BFS_ERR_INVALID;
    }
    bfs_status s = ensure_ms(g, 0);
    if (s != BFS_OK) return s;
    cudaStream_t st = as_stream(stream);
    bfs_batch_config base = g->ms->cfg;
    base.timing = 0;
    cudaEvent_t e0, e1;
    GB_CK(cudaEventCreate(&e0));
    GB_CK(cudaEventCreate(&e1));
    auto timed = [&](const bfs_batch_config &c, float *ms) -> bfs_status {
        g->ms->cfg = c;
        bfs_status r = bfs_run_batch(g, roots, k, levels_scratch, stream);  // warm
        if (r != BFS_OK) return r;
        float best_t = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            GB_CK(cudaEventRecord(e0, st));
            r = bfs_run_batch(g, roots, k, levels_scratch, stream);
            if (r != BFS_OK) return r;
            GB_CK(cudaEventRecord(e1, st));
            GB_CK(cudaEventSynchronize(e1));
            float t = 0;
            GB_CK(cudaEventElapsedTime(&t, e0, e1));
            best_t = std::min(best_t, t);
        }
        *ms = best_t;
        return BFS_OK;
    };
    // Coordinate search: alpha, then beta, then the lane probe length.
    bfs_batch_config cur = base;
    float cur_t = 0;
    if ((s = timed(cur, &cur_t)) != BFS_OK) goto done;
    {
        const double alphas[] = {1.0, 2.0, 4.0, 8.0, 14.0, 32.0, 128.0};
        const double betas[] = {6.0, 24.0, 96.0, 1e9};
        const int probes[] = {4, 16, 64, 256};
        for (double a : alphas) {
            bfs_batch_config c = cur;
            c.alpha = a;
            float t;
            if ((s = timed(c, &t)) != BFS_OK) goto done;
            if (t < cur_t) { cur = c; cur_t = t; }
        }
        for (double b : betas) {
            bfs_batch_config c = cur;
            c.beta = b;
            float t;
            if ((s = timed(c, &t)) != BFS_OK) goto done;
            if (t < cur_t) { cur = c; cur_t = t; }
        }
        for (int p : probes) {
            bfs_batch_config c = cur;
            c.lane_probe = p;
            float t;
            if ((s = timed(c, &t)) != BFS_OK) goto done;
            if (t < cur_t) { cur = c; cur_t = t; }
        }
        {  // host-driven layers or the device-side loop in one graph
            bfs_batch_config c = cur;
            c.use_graph = !cur.use_graph;
            float t;
            if ((s = timed(c, &t)) != BFS_OK) goto done;
            if (t < cur_t) { cur = c; cur_t = t; }
        }
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cur.timing = base.timing;
    g->ms->cfg = (s == BFS_OK) ? cur : base;
    if (s == BFS_OK && best) *best = cur;
    return s;
}

extern "C" BFS_API bfs_status bfs_selftest_grid_barrier(int32_t missing_blocks, int64_t timeout_us,
                                                        void *stream) {
    clear_error();
    if (missing_blocks < 0 || missing_blocks > 1024 || timeout_us < 1000 ||
        timeout_us > 10000000) {
        set_error("bfs_selftest_grid_barrier: need 0 <= missing <= 1024 and 1 ms <= timeout <= 10 s");
        return BFS_ERR_INVALID;
    }
    cudaStream_t st = as_stream(stream);
    int32_t *buf = nullptr;  // bar[2], err, ok
    GB_CK(dev_malloc_async(&buf, 16, st));
    const int32_t init[4] = {0, 0, 0, 1};
    int32_t out[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(buf, init, 16, cudaMemcpyHostToDevice, st);
    const unsigned missing = (unsigned)missing_blocks;
    unsigned long long tns = (unsigned long long)timeout_us * 1000ull;
    unsigned *bar = (unsigned *)buf;
    int32_t *err = buf + 2, *ok = buf + 3;
    void *args[] = {&bar, &err, (void *)&missing, &tns, &ok};
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((const void *)barrier_probe_kernel, dim3(sm_count()),
                                        dim3(32), args, 0, st);
    count_launch();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, buf, 16, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(buf, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "barrier self-test", __FILE__, __LINE__);
    if (e2 != cudaSuccess) return cuda_status(e2, "barrier self-test", __FILE__, __LINE__);
    if (!out[3]) {
        set_error("grid barrier wait ran out after %lld us (%d blocks never arrived)",
                  (long long)timeout_us, missing_blocks);
        return BFS_ERR_TIMEOUT;
    }
    return BFS_OK;
}
