// bfs.cu -- single-source hybrid BFS (Alg. 1-3, Sec. 5) on one GPU.
//
// Data on the device, per graph:
//   off[n+1] int64, idx[nnz] int32            symmetric CSR, rows sorted
//   visited, front, next : uint32[nw_pad]      n-bit bitmaps (Sec. 5.1 "vis",
//                                              "in", "out"); words past n are
//                                              marked visited
//   q_a, q_b : int32[n]                        frontier queues for top-down
//   big : int32[n]                             frontier vertices whose edges
//                                              are spread over the whole grid
//   trace : int64[kRing][8]                    per-layer counters (Sec. 4)
//
// One layer = one of
//   top-down  (Alg. 1): td_kernel over the queue, vertices binned by degree
//             (shared-warp gather below td_warp_degree, one warp per vertex
//             below td_grid_degree), then td_big_kernel spreads the edges of
//             the big vertices over the grid. A vertex is claimed by
//             atomicCAS on its parent; the winner writes its level, sets its
//             visited / next bits and appends it to the next queue.
//   bottom-up (Alg. 2 / Sec. 5.1): bu_kernel, one warp per 32-vertex bitmap
//             word, one lane per vertex. Each unvisited lane tests its first
//             bu_probe neighbours itself (the MAX_POS probe of Sec. 5.2); the
//             lanes still unresolved are then scanned by the whole warp, 32
//             neighbours per step, __ballot_sync + __ffs picking the first
//             frontier neighbour in CSR order. The warp owns the word, so the
//             next / visited words are written without atomics.
// and the switch counters v_f, e_f (plus edges examined) are reduced inside
// the step kernels into the layer's trace slot. The host reads that slot after
// each layer and applies the Alg. 3 switch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

#include "graph.cuh"

namespace gbfs {
namespace {

// Read-only loads of data that is constant within one launch of the
// host-driven loop but written by other blocks earlier in a persistent launch.
template <bool CO, typename T>
__device__ __forceinline__ T ldro(const T *p) {
    if constexpr (CO) return __ldcg(p);
    else return __ldg(p);
}

__device__ __forceinline__ int64_t deg_of(const int64_t *__restrict__ off, int32_t v) {
    return off[v + 1] - off[v];
}

// Marks, per bitmap word, the vertices no traversal can reach from another
// vertex: degree 0 (no edge leads to them) and ids past n (padding).
__global__ void base_vis_kernel(const int64_t *__restrict__ off, int64_t n, int64_t nw_pad,
                                uint32_t *__restrict__ base) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw_pad; w += stride) {
        uint32_t bits = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t v = w * 32 + b;
            if (v >= n || off[v + 1] == off[v]) bits |= 1u << b;
        }
        base[w] = bits;
    }
}

// Per-vertex head record for the bottom-up probe: the first entry of the
// vertex's CSR row (-1 if it has none) and the degree.
__global__ void head_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                            int64_t n, int2 *__restrict__ head) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t b = off[v];
        const int d = (int)(off[v + 1] - b);
        head[v] = make_int2(d > 0 ? idx[b] : -1, d);
    }
}

// Hub head record: the neighbour of largest degree (smallest id on ties, -1
// if none) and the degree. One warp per vertex; the lanes stride over the row
// and a warp max of degree << 32 | ~id picks the hub.
__global__ void hub_head_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                                int64_t n, int2 *__restrict__ head) {
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = gw; v < n; v += tw) {
        const int64_t b = off[v], e = off[v + 1];
        unsigned long long best = 0;
        for (int64_t q = b + lane; q < e; q += 32) {
            const int32_t u = idx[q];
            const unsigned long long du = (unsigned long long)(off[u + 1] - off[u]);
            const unsigned long long key = du << 32 | (unsigned long long)(~(uint32_t)u);
            best = key > best ? key : best;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other > best ? other : best;
        }
        if (lane == 0)
            head[v] = make_int2(e > b ? (int32_t)(~(uint32_t)(best & 0xffffffffull)) : -1,
                                (int)(e - b));
    }
}

// Exclusive prefix count of the degree >= 1 vertices per bitmap word:
// wrank[w] = set bits of ~base in words 0..w-1, wrank[nw_pad] = the total.
// One block walks the words 1024 at a time (once per graph).
__global__ void __launch_bounds__(1024) word_rank_kernel(const uint32_t *__restrict__ base,
                                                         int64_t nw_pad,
                                                         uint32_t *__restrict__ wrank) {
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t b = 0; b < nw_pad; b += 1024) {
        const int64_t w = b + threadIdx.x;
        const uint32_t c = w < nw_pad ? (uint32_t)__popc(~base[w]) : 0u;
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            const uint32_t t = warp_tot[lane];
            uint32_t sc = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, sc, o);
                if ((int)lane >= o) sc += y;
            }
            warp_tot[lane] = sc - t;
        }
        __syncthreads();
        if (w < nw_pad) wrank[w] = carry + warp_tot[wid] + x - c;
        __syncthreads();
        if (threadIdx.x == 1023) carry += warp_tot[wid] + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) wrank[nw_pad] = carry;
}

// Compact hub records: for every degree >= 1 vertex v (a clear bit of
// base), hubc[rank(v)] = hub | (degree == 1) << 31, rank(v) = wrank[w] +
// the degree >= 1 vertices before v in its word. A warp per word.
__global__ void hubc_kernel(const int2 *__restrict__ head, const uint32_t *__restrict__ base,
                            const uint32_t *__restrict__ wrank, int64_t nw_pad,
                            uint32_t *__restrict__ hubc) {
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = gw; w < nw_pad; w += tw) {
        const uint32_t live = ~base[w];
        if ((live >> lane) & 1u) {
            const int2 h = head[w * 32 + lane];
            hubc[wrank[w] + __popc(live & lanemask_lt())] =
                (uint32_t)h.x | (h.y == 1 ? 0x80000000u : 0u);
        }
    }
}

// {base word, rank} per bitmap word, the streaming sweep's per-word metadata.
__global__ void wmeta_kernel(const uint32_t *__restrict__ base, const uint32_t *__restrict__ wrank,
                             int64_t nw_pad, uint2 *__restrict__ wmeta) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw_pad; w += stride)
        wmeta[w] = make_uint2(base[w], wrank[w]);
}

// Highest-degree vertex (smallest id on ties), packed as degree << 32 | ~id.
__global__ void max_degree_kernel(const int64_t *__restrict__ off, int64_t n,
                                  unsigned long long *best) {
    unsigned long long b = 0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long d = (unsigned long long)(off[v + 1] - off[v]);
        const unsigned long long key = (d << 32) | (0xffffffffull - (unsigned long long)v);
        b = key > b ? key : b;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, b, o);
        b = y > b ? y : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(best, b);
}

// Bitmap of the vertices a traversal reached (level >= 0).
__global__ void reached_bits_kernel(const int32_t *__restrict__ level, int64_t n, int64_t nw_pad,
                                    uint32_t *__restrict__ bits) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw_pad; w += stride) {
        uint32_t x = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t v = w * 32 + b;
            if (v < n && level[v] >= 0) x |= 1u << b;
        }
        bits[w] = x;
    }
}

// write_out = 0 leaves level and parent unwritten except at the root: the
// first hub sweep of the traversal (or out_fill_kernel) writes the rest.
__global__ void init_kernel(int64_t n, int64_t nw_pad, int32_t root,
                            const int64_t *__restrict__ off, const uint32_t *__restrict__ base,
                            const uint32_t *__restrict__ comp_in,
                            int32_t *__restrict__ level, int32_t *__restrict__ parent,
                            uint32_t *__restrict__ visited, uint32_t *__restrict__ front,
                            int32_t *__restrict__ queue, int64_t *__restrict__ trace,
                            int write_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (write_out) {
        for (int64_t i = t0; i < n; i += stride) {
            level[i] = (i == root) ? 0 : -1;
            parent[i] = (i == root) ? root : -1;
        }
    } else if (t0 == 0) {
        level[root] = 0;
        parent[root] = root;
    }
    const int64_t rw = root >> 5;
    const uint32_t rbit = 1u << (root & 31);
    // with a component mask that holds the root, everything outside it
    // starts visited: no edge leads there from the root
    const bool prune = comp_in && ((comp_in[rw] & rbit) != 0u);
    for (int64_t w = t0; w < nw_pad; w += stride) {
        visited[w] = base[w] | (w == rw ? rbit : 0u) | (prune ? ~comp_in[w] : 0u);
        front[w] = (w == rw) ? rbit : 0u;
    }
    for (int64_t i = t0; i < kRing * kFields; i += stride) {
        int64_t v = 0;
        if (i == T_NF) v = 1;
        if (i == T_MF) v = deg_of(off, root);
        trace[i] = v;
    }
    if (t0 == 0) queue[0] = root;
}

// Copies a trace slot into the mapped host block and then, after a system
// fence, the sequence number the host waits for (one thread: the counters
// are final, the kernels that added them came before on the stream).
__global__ void publish_kernel(const int64_t *__restrict__ slot, int64_t *pub, int64_t seq) {
    if (threadIdx.x == 0) {
        volatile int64_t *vp = pub;
        for (int i = 0; i < kFields; ++i) vp[i] = slot[i];
        __threadfence_system();
        vp[kFields] = seq;
    }
}

// Clears *flag when some CSR row is not in ascending order (thread per row).
__global__ void rows_sorted_kernel(const int64_t *__restrict__ off,
                                   const int32_t *__restrict__ idx, int64_t n, int *flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t b = off[v], e = off[v + 1];
        for (int64_t q = b + 1; q < e; ++q)
            if (idx[q] < idx[q - 1]) {
                atomicExch(flag, 0);
                break;
            }
    }
}

// Smallest-id parent one level up for every reached vertex other than the
// root (parent_min); a vertex at level 1 takes the root, the only vertex at
// level 0. A lane per vertex tests the first P row entries itself,
// B at a time (B index loads, then B level loads, all independent); rows
// still open after P entries are finished by the whole warp, 32 entries per
// round. With ascending rows the first neighbour at level - 1 is the
// smallest and ends the scan; otherwise the whole row is scanned for the
// minimum.
__global__ void __launch_bounds__(kBlock) min_parent_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
    const int32_t *__restrict__ level, int32_t *__restrict__ parent, int64_t n, int32_t root,
    int sorted) {
    constexpr int P = 32, B = 8;
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = gw; w < (n + 31) / 32; w += tw) {
        const int64_t v = w * 32 + lane;
        const int32_t lv = v < n ? level[v] : -1;
        const bool active = v < n && v != root && lv > 0;
        int64_t b = 0, e = 0;
        if (active) {
            b = off[v];
            e = off[v + 1];
        }
        // level 1: the root is the only vertex one level up (no scan; a hub
        // next to the root would otherwise scan its row up to the root's id)
        int32_t best = active && lv == 1 ? root : 0x7fffffff;
        bool done = !active || lv == 1;
        for (int q0 = 0; q0 < P; q0 += B) {
            if (done || b + q0 >= e) break;
            int32_t u[B], lu[B];
#pragma unroll
            for (int t = 0; t < B; ++t) u[t] = b + q0 + t < e ? __ldg(idx + b + q0 + t) : -1;
#pragma unroll
            for (int t = 0; t < B; ++t) lu[t] = u[t] >= 0 ? __ldg(level + u[t]) : -2;
#pragma unroll
            for (int t = 0; t < B; ++t)
                if (!done && lu[t] == lv - 1) {  // lv - 1 >= 0, so u[t] >= 0 here
                    best = u[t] < best ? u[t] : best;
                    if (sorted) done = true;
                }
        }
        unsigned pend = __ballot_sync(0xffffffffu, !done && e - b > P);
        while (pend) {
            const int L = __ffs(pend) - 1;
            pend &= pend - 1;
            const int64_t lb = __shfl_sync(0xffffffffu, b, L) + P;
            const int64_t le = __shfl_sync(0xffffffffu, e, L);
            const int32_t want = __shfl_sync(0xffffffffu, lv, L) - 1;
            int32_t bL = __shfl_sync(0xffffffffu, best, L);
            for (int64_t q0 = lb; q0 < le; q0 += 32) {
                const int64_t q = q0 + lane;
                const int32_t u = q < le ? __ldg(idx + q) : 0x7fffffff;
                const bool hit = q < le && __ldg(level + u) == want;
                int32_t c = hit ? u : 0x7fffffff;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const int32_t y = __shfl_xor_sync(0xffffffffu, c, o);
                    c = y < c ? y : c;
                }
                bL = c < bL ? c : bL;
                if (sorted && __ballot_sync(0xffffffffu, hit)) break;
            }
            if ((int)lane == L) best = bL;
        }
        if (active) parent[v] = best;
    }
}

// level = parent = -1 for every vertex not reached so far (not visited, or
// visited only as a degree-0 vertex or id past n), the root excepted: the
// outputs of a traversal that started without write_out and has had no
// writing hub sweep.
__device__ __forceinline__ void out_fill_phase(int64_t n, int32_t root,
                                               const uint32_t *__restrict__ visited,
                                               const uint32_t *__restrict__ base,
                                               int32_t *__restrict__ level,
                                               int32_t *__restrict__ parent) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        const uint32_t reached = visited[v >> 5] & ~base[v >> 5];
        if (v != root && !((reached >> (v & 31)) & 1u)) {
            if (level) level[v] = -1;
            parent[v] = -1;
        }
    }
}

__global__ void out_fill_kernel(int64_t n, int32_t root, const uint32_t *__restrict__ visited,
                                const uint32_t *__restrict__ base,
                                int32_t *__restrict__ level, int32_t *__restrict__ parent) {
    out_fill_phase(n, root, visited, base, level, parent);
}

// Level pass: the levels of a traversal whose layers kept their frontier
// bitmaps in a ring (slot j = the vertices of level j, j < slots <= 16):
// vertex v gets the j whose slot holds it, or -1 when no slot does (each
// vertex is in at most one). A warp covers 8 consecutive words per round:
// lane j loads slot j's 8 words (two 16-byte loads); for each word, OR
// reductions over the lanes give the union of the slots and the 4 bit planes
// of j (plane p = OR of the slots whose j has bit p), from which lane i reads
// vertex i's level; the level stores are whole 128-byte rows.
static_assert(kLevelRing <= 16, "the level pass reads levels as 4 bit planes");
__global__ void level_pass_kernel(const uint32_t *__restrict__ ring, int64_t nw_pad, int slots,
                                  int64_t n, int32_t *__restrict__ level) {
    constexpr int R = 8;
    static_assert(32 % R == 0, "a round's R words must not cross nw_pad (a multiple of 32)");
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w0 = gw * R; w0 < nw_pad && w0 * 32 < n; w0 += tw * R) {
        uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
        if ((int)lane < slots) {
            const uint4 *src = reinterpret_cast<const uint4 *>(ring + (int64_t)lane * nw_pad + w0);
            lo = __ldg(src);
            hi = __ldg(src + 1);
        }
        const uint32_t x[R] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t any = __reduce_or_sync(0xffffffffu, x[k]);
            const uint32_t p0 = __reduce_or_sync(0xffffffffu, (lane & 1u) ? x[k] : 0u);
            const uint32_t p1 = __reduce_or_sync(0xffffffffu, (lane & 2u) ? x[k] : 0u);
            const uint32_t p2 = __reduce_or_sync(0xffffffffu, (lane & 4u) ? x[k] : 0u);
            const uint32_t p3 = __reduce_or_sync(0xffffffffu, (lane & 8u) ? x[k] : 0u);
            const int lv = ((any >> lane) & 1u)
                               ? (int)(((p0 >> lane) & 1u) | (((p1 >> lane) & 1u) << 1) |
                                       (((p2 >> lane) & 1u) << 2) | (((p3 >> lane) & 1u) << 3))
                               : -1;
            const int64_t v = (w0 + k) * 32 + lane;
            if (v < n) __stcs(level + v, lv);
        }
    }
}

__device__ __forceinline__ void block_add4(int64_t a, int64_t b, int64_t c, int64_t e,
                                           unsigned long long *dst_a,
                                           unsigned long long *dst_b,
                                           unsigned long long *dst_c,
                                           unsigned long long *dst_e) {
    __shared__ long long red[4][kBlock / 32];
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    e = warp_sum(e);
    const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][w] = a;
        red[1][w] = b;
        red[2][w] = c;
        red[3][w] = e;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            s0 += red[0][i];
            s1 += red[1][i];
            s2 += red[2][i];
            s3 += red[3][i];
        }
        if (dst_a && s0) atomicAdd(dst_a, (unsigned long long)s0);
        if (dst_b && s1) atomicAdd(dst_b, (unsigned long long)s1);
        if (dst_c && s2) atomicAdd(dst_c, (unsigned long long)s2);
        if (dst_e && s3) atomicAdd(dst_e, (unsigned long long)s3);
    }
}

__device__ __forceinline__ void block_add3(int64_t a, int64_t b, int64_t c,
                                           unsigned long long *dst_a,
                                           unsigned long long *dst_b,
                                           unsigned long long *dst_c) {
    block_add4(a, b, c, 0, dst_a, dst_b, dst_c, nullptr);
}

// State shared by the top-down expansion paths.
struct TdArgs {
    const int64_t *__restrict__ off;
    const int32_t *__restrict__ idx;
    uint32_t *visited;
    uint32_t *next_bm;
    int32_t *parent;
    int32_t *level;
    int32_t *q_next;
    unsigned long long *next_count;  // trace slot of the next layer, T_NF
    int32_t new_level;
    int queue_mode;  // 1: append winners to q_next; 0: next bitmap only
    int claim;       // 0: atomicCAS on parent; 1: atomicOr on the visited word
    int defer;       // 1: a winner stores only its parent and next bit; its
                     // level and the n_f / m_f counts come from td_post
};

// K edges (u[k], v[k]) per lane of the top-down step (the inner loop of Alg. 1),
// called by all 32 lanes together; valid[k] masks missing edges. The visited
// bitmap (L2-resident) filters first. The claim is either the CAS of
// parent[v] from -1 to u (claim 0), or a fetch-or of v's bit into its
// visited word (claim 1: an L2 atomic instead of a read-modify-write of the
// parent array in HBM), after which the winner stores parent[v] = u. The K
// loads and the K atomics of a lane are issued back to back. A winner writes
// its level, sets its visited and next bits, and adds its degree to mf and 1
// to nf. In queue mode winners are appended to the next queue with one
// atomicAdd per warp and edge slot.
template <int K>
__device__ __forceinline__ void td_visit(const TdArgs &a, const bool (&valid)[K],
                                         const int32_t (&u)[K], const int32_t (&v)[K],
                                         int64_t &mf, int64_t &nf) {
    uint32_t vw[K];
#pragma unroll
    for (int k = 0; k < K; ++k) vw[k] = valid[k] ? __ldcg(a.visited + (v[k] >> 5)) : 0xffffffffu;
    bool won[K];
    if (a.claim == 0) {
        int old[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool cand = valid[k] && !((vw[k] >> (v[k] & 31)) & 1u);
            old[k] = cand ? atomicCAS(a.parent + v[k], -1, u[k]) : 0;
            won[k] = cand && old[k] == -1;
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (won[k]) atomicOr(a.visited + (v[k] >> 5), 1u << (v[k] & 31));
    } else {
        uint32_t old[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t bit = 1u << (v[k] & 31);
            const bool cand = valid[k] && !(vw[k] & bit);
            old[k] = cand ? atomicOr(a.visited + (v[k] >> 5), bit) : 0xffffffffu;
            won[k] = cand && !(old[k] & bit);
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (won[k]) a.parent[v[k]] = u[k];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (won[k]) {
            atomicOr(a.next_bm + (v[k] >> 5), 1u << (v[k] & 31));
            if (!a.defer) {
                if (a.level) a.level[v[k]] = a.new_level;
                mf += deg_of(a.off, v[k]);
                nf += 1;
            }
        }
    }
    if (a.queue_mode) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const unsigned wm = __ballot_sync(0xffffffffu, won[k]);
            if (wm) {
                const int leader = __ffs(wm) - 1;
                unsigned long long base = 0;
                if ((int)lane_id() == leader)
                    base = atomicAdd(a.next_count, (unsigned long long)__popc(wm));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (won[k]) a.q_next[base + __popc(wm & lanemask_lt())] = v[k];
            }
        }
    }
}

// Top-down over the frontier queue. A warp takes `per_warp` (1..32) queue
// entries, one per lane, and splits them by degree: >= grid_deg go to the big
// list (td_big_kernel), >= warp_deg are expanded one at a time by the whole
// warp (64 edges per round), the rest are gathered together: a warp-wide
// exclusive scan of their degrees gives each lane two edges per round.
template <bool CO>
__device__ __forceinline__ void td_phase(TdArgs a, const int32_t *__restrict__ q,
                                                    int64_t qlen, int per_warp,
                                                    int32_t *__restrict__ big,
                                                    unsigned long long *big_count,
                                                    unsigned long long *next_mf, int warp_deg,
                                                    int64_t grid_deg, int64_t *zero_slot) {
    if (blockIdx.x == 0 && threadIdx.x < kFields) zero_slot[threadIdx.x] = 0;
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t my_mf = 0, my_nf = 0;
    for (int64_t base = gw * per_warp; base < qlen; base += tw * per_warp) {
        const int64_t i = base + lane;
        const bool have = (int)lane < per_warp && i < qlen;
        int32_t u = 0;
        int64_t beg = 0, end = 0;
        if (have) {
            u = ld<CO>(q + i);
            beg = a.off[u];
            end = a.off[u + 1];
        }
        const int64_t deg = end - beg;
        const bool isbig = have && deg >= grid_deg;
        const unsigned bm = __ballot_sync(0xffffffffu, isbig);
        if (bm) {
            const int leader = __ffs(bm) - 1;
            unsigned long long b0 = 0;
            if ((int)lane == leader) b0 = atomicAdd(big_count, (unsigned long long)__popc(bm));
            b0 = __shfl_sync(0xffffffffu, b0, leader);
            if (isbig) big[b0 + __popc(bm & lanemask_lt())] = u;
        }
        const bool isw = have && !isbig && deg >= warp_deg;
        unsigned wm = __ballot_sync(0xffffffffu, isw);
        while (wm) {
            const int L = __ffs(wm) - 1;
            wm &= wm - 1;
            const int32_t lu = __shfl_sync(0xffffffffu, u, L);
            const int64_t lb = __shfl_sync(0xffffffffu, beg, L);
            const int64_t le = __shfl_sync(0xffffffffu, end, L);
            for (int64_t e0 = lb; e0 < le; e0 += 32 * kTdK) {
                bool ok[kTdK];
                int32_t uu[kTdK], vv[kTdK];
#pragma unroll
                for (int k = 0; k < kTdK; ++k) {
                    const int64_t e = e0 + 32 * k + lane;
                    ok[k] = e < le;
                    uu[k] = lu;
                    vv[k] = ok[k] ? a.idx[e] : 0;
                }
                td_visit<kTdK>(a, ok, uu, vv, my_mf, my_nf);
            }
        }
        const int sdeg = (have && !isbig && !isw) ? (int)deg : 0;
        int total;
        const int excl = warp_exclusive_scan(sdeg, &total);
        for (int j0 = 0; j0 < total; j0 += 64) {
            bool ok[2];
            int32_t uu[2], vv[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int j = j0 + 32 * k + (int)lane;
                // owner = the last lane whose exclusive prefix is <= j
                int lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int ex = __shfl_sync(0xffffffffu, excl, lo + step);
                    if (ex <= j) lo += step;
                }
                uu[k] = __shfl_sync(0xffffffffu, u, lo);
                const int64_t ob = __shfl_sync(0xffffffffu, beg, lo);
                const int oex = __shfl_sync(0xffffffffu, excl, lo);
                ok[k] = j < total;
                vv[k] = ok[k] ? a.idx[ob + (j - oex)] : 0;
            }
            td_visit<2>(a, ok, uu, vv, my_mf, my_nf);
        }
    }
    block_add3(my_mf, a.queue_mode ? 0 : my_nf, 0, next_mf, a.next_count, nullptr);
}

__global__ void __launch_bounds__(kBlock) td_kernel(TdArgs a, const int32_t *__restrict__ q,
                                                    int64_t qlen, int per_warp,
                                                    int32_t *__restrict__ big,
                                                    unsigned long long *big_count,
                                                    unsigned long long *next_mf, int warp_deg,
                                                    int64_t grid_deg, int64_t *zero_slot) {
    td_phase<false>(a, q, qlen, per_warp, big, big_count, next_mf, warp_deg, grid_deg, zero_slot);
}


// The edges of all big vertices, spread evenly over the grid: batches of
// kBigBatch vertices, an exclusive scan of their degrees in shared memory,
// then a grid-stride walk over the batch's edge range (64 edges per warp and
// round) with a binary search for the owning vertex.
template <bool CO>
__device__ __forceinline__ void td_big_phase(TdArgs a, const int32_t *__restrict__ big,
                                                        const unsigned long long *big_count,
                                                        unsigned long long *next_mf) {
    __shared__ long long pre[kBigBatch + 1];
    __shared__ long long beg_s[kBigBatch];
    __shared__ int32_t u_s[kBigBatch];
    __shared__ long long wtot[kBlock / 32];
    const int64_t cnt = (int64_t)ld<CO>(big_count);
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    constexpr int per = kBigBatch / kBlock;
    int64_t my_mf = 0, my_nf = 0;
    for (int64_t b0 = 0; b0 < cnt; b0 += kBigBatch) {
        const int nb = (int)(cnt - b0 < kBigBatch ? cnt - b0 : kBigBatch);
        long long dsum = 0;
        long long dloc[per];
#pragma unroll
        for (int k = 0; k < per; ++k) {
            const int t = threadIdx.x * per + k;
            long long d = 0;
            if (t < nb) {
                const int32_t u = ld<CO>(big + b0 + t);
                u_s[t] = u;
                beg_s[t] = a.off[u];
                d = a.off[u + 1] - beg_s[t];
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
        if (threadIdx.x == kBlock - 1) pre[kBigBatch] = run;
        __syncthreads();
        const long long total = pre[kBigBatch];
        for (long long g0 = gw * 32 * kTdK; g0 < total; g0 += tw * 32 * kTdK) {
            // Owner of the round's first edge by one binary search (the last
            // j in [0, nb) with pre[j] <= g0), then each lane walks forward:
            // every listed vertex has at least 4 * td_warp_degree edges, so a
            // round's 32 * kTdK edges cross at most a couple of row ends.
            int lo = 0;
            {
                int hi = nb;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (pre[mid] <= g0) lo = mid;
                    else hi = mid;
                }
            }
            bool ok[kTdK];
            int32_t uu[kTdK], vv[kTdK];
#pragma unroll
            for (int k = 0; k < kTdK; ++k) {
                const long long g = g0 + 32 * k + lane;
                ok[k] = g < total;
                uu[k] = 0;
                vv[k] = 0;
                if (ok[k]) {
                    while (lo + 1 < nb && pre[lo + 1] <= g) ++lo;
                    uu[k] = u_s[lo];
                    vv[k] = a.idx[beg_s[lo] + (g - pre[lo])];
                }
            }
            td_visit<kTdK>(a, ok, uu, vv, my_mf, my_nf);
        }
        __syncthreads();
    }
    block_add3(my_mf, a.queue_mode ? 0 : my_nf, 0, next_mf, a.next_count, nullptr);
}

__global__ void __launch_bounds__(kBlock) td_big_kernel(TdArgs a, const int32_t *__restrict__ big,
                                                        const unsigned long long *big_count,
                                                        unsigned long long *next_mf) {
    td_big_phase<false>(a, big, big_count, next_mf);
}

// A bitmap-output top-down layer defers its winners' level stores and
// counts to td_post when the vertices it can still find (unvisited, degree
// > 0) outnumber the bitmap words; with fewer, one random store per winner
// costs less than a pass over the bitmap.
__host__ __device__ inline int td_defer(int queue_mode, int64_t findable, int64_t nw) {
    return !queue_mode && findable >= nw ? 1 : 0;
}

// Completes a deferred top-down layer from its next bitmap: level = d+1 for
// every new frontier vertex, and the counters n_f (popcount) and m_f (degree
// sum) of the next layer. A warp takes 8 words per round and lane i handles
// bit i of each, so the level stores and row-bound loads are coalesced
// instead of one random sector per winner.
template <bool CO>
__device__ __forceinline__ void td_post_phase(const int64_t *__restrict__ off,
                                              const uint32_t *__restrict__ next, int64_t nw,
                                              int32_t *__restrict__ level, int32_t new_level,
                                              unsigned long long *next_nf,
                                              unsigned long long *next_mf) {
    // A warp takes 32 words per round (one coalesced load, lane i word i)
    // and then gives each lane one of the round's set bits at a time: lane j
    // finds the word holding the j-th set bit by a binary search over the
    // lanes' exclusive bit counts (shuffles) and the bit by halving popcounts.
    // The row bounds of up to 32 found vertices are then loaded together.
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t my_nf = 0, my_mf = 0;
    for (int64_t w0 = gw * 32; w0 < nw; w0 += tw * 32) {
        const uint32_t x = w0 + lane < nw ? ld<CO>(next + w0 + lane) : 0u;
        const int cnt = __popc(x);
        int tot;
        const int excl = warp_exclusive_scan(cnt, &tot);
        my_nf += cnt;
        for (int base = 0; base < tot; base += 32) {
            const int j = base + (int)lane;
            int owner = 0;  // the last lane whose exclusive count is <= j
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int cand = owner + step;
                const int ec = __shfl_sync(0xffffffffu, excl, cand & 31);
                if (cand < 32 && ec <= j) owner = cand;
            }
            const uint32_t xo = __shfl_sync(0xffffffffu, x, owner);
            const int eo = __shfl_sync(0xffffffffu, excl, owner);
            if (j < tot) {
                // position of set bit number r of xo
                uint32_t m = xo;
                int r = j - eo, pos = 0;
#pragma unroll
                for (int h = 16; h > 0; h >>= 1) {
                    const int c = __popc(m & ((1u << h) - 1u));
                    if (r >= c) {
                        r -= c;
                        m >>= h;
                        pos += h;
                    }
                }
                const int64_t v = (w0 + owner) * 32 + pos;
                my_mf += off[v + 1] - off[v];
                if (level) level[v] = new_level;
            }
        }
    }
    block_add3(my_nf, my_mf, 0, next_nf, next_mf, nullptr);
}

__global__ void __launch_bounds__(kBlock) td_post_kernel(const int64_t *__restrict__ off,
                                                         const uint32_t *__restrict__ next,
                                                         int64_t nw, int32_t *__restrict__ level,
                                                         int32_t new_level,
                                                         unsigned long long *next_nf,
                                                         unsigned long long *next_mf) {
    td_post_phase<false>(off, next, nw, level, new_level, next_nf, next_mf);
}


// Bottom-up step (Alg. 2 with the Sec. 5.1 structure). Lane-per-vertex,
// warp-per-word: a warp takes a chunk of 32 consecutive bitmap words (their
// visited words loaded together) and walks it W words at a time, so W
// independent word-tasks are in flight per warp. Per word and lane:
//   1. the lane's own probe of its first `probe` neighbours, CH independent
//      index loads then CH frontier-bit loads per round (the MAX_POS probe of
//      Sec. 5.2; the 16-lane gather of Alg. 5 recast for 32 lanes);
//   2. the rows still unresolved are scanned by the whole warp, 64
//      neighbours per round, __ballot_sync + __ffs selecting the first
//      frontier neighbour in CSR order (Alg. 2 stops at the first hit);
//   3. the ballot of found lanes is the next word and is ORed into the
//      visited word by the owning warp, without atomics.
// Row positions are 32-bit offsets from a per-lane row pointer. With HEAD the
// first probe and the degree come from the vertex's 8-byte head record (one
// coalesced load per lane) and the row bound is read only after that probe
// misses. hskip says where the row scan then starts: 1 when the record holds
// the row's first entry (already tested), 0 when it holds the hub.
template <int W, int CH, bool HEAD, bool CO>
__device__ __forceinline__ void bu_phase(
    const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
    const int2 *__restrict__ head, int64_t nw_pad,
    uint32_t *__restrict__ visited, const uint32_t *__restrict__ front,
    uint32_t *__restrict__ next_bm, int32_t *__restrict__ parent, int32_t *__restrict__ level,
    int32_t new_level, int probe, unsigned long long *slot_next, int64_t *zero_slot, int span,
    int hskip) {
    if (blockIdx.x == 0 && threadIdx.x < kFields) zero_slot[threadIdx.x] = 0;
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = nw_pad >> 5;
    // a warp task is `span` consecutive words of a 32-word chunk (span = 32
    // on large graphs; smaller on small ones so every warp gets work)
    const int per = 32 / span;
    const int64_t ntasks = nchunks * per;
    int64_t my_nf = 0, my_mf = 0, my_ex = 0;
    for (int64_t t = gw; t < ntasks; t += tw) {
        const int64_t c = t / per;
        const int j0 = (int)(t - c * per) * span;
        const uint32_t vis_lane = ld<CO>(visited + c * 32 + lane);
        uint32_t *const next_c = next_bm + c * 32;
        uint32_t *const vis_c = visited + c * 32;
        const int64_t v_c = c * 1024 + lane;
        for (int j = j0; j < j0 + span; j += W) {
            uint32_t vw[W];
            bool all = true;
#pragma unroll
            for (int k = 0; k < W; ++k) {
                vw[k] = __shfl_sync(0xffffffffu, vis_lane, j + k);
                all = all && vw[k] == 0xffffffffu;
            }
            if (all) {
                if ((int)lane < W) next_c[j + lane] = 0u;
                continue;
            }
            bool unv[W], found[W];
            const int32_t *row[W];
            int deg[W], ex[W];
            int32_t p[W];
            // positions [0, lane_lim) are tested by the lane itself
            const int lane_lim = HEAD ? (probe > hskip ? probe : hskip) : probe;
            if (HEAD) {
                int2 h[W];
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    const int64_t v = v_c + (j + k) * 32;
                    unv[k] = !((vw[k] >> lane) & 1u);  // bits past n are set
                    found[k] = false;
                    p[k] = -1;
                    ex[k] = 0;
                    h[k] = unv[k] ? __ldg(head + v) : make_int2(-1, 0);
                    deg[k] = h[k].y;
                    row[k] = idx;
                }
                uint32_t fw[W];
#pragma unroll
                for (int k = 0; k < W; ++k) fw[k] = h[k].x >= 0 ? ldro<CO>(front + (h[k].x >> 5)) : 0u;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    if (h[k].x >= 0) {
                        ex[k] = 1;
                        if ((fw[k] >> (h[k].x & 31)) & 1u) {
                            found[k] = true;
                            p[k] = h[k].x;
                        }
                    }
                    if (unv[k] && !found[k] && deg[k] > hskip)
                        row[k] = idx + off[v_c + (j + k) * 32];
                }
            } else {
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    const int64_t v = v_c + (j + k) * 32;
                    unv[k] = !((vw[k] >> lane) & 1u);  // bits past n are set
                    found[k] = false;
                    p[k] = -1;
                    ex[k] = 0;
                    int64_t b = 0, e = 0;
                    if (unv[k]) {
                        b = off[v];
                        e = off[v + 1];
                    }
                    row[k] = idx + b;
                    deg[k] = (int)(e - b);
                }
            }
            for (int p0 = HEAD ? hskip : 0; p0 < lane_lim; p0 += CH) {
                int32_t cand[W][CH];
                bool any = false;
#pragma unroll
                for (int k = 0; k < W; ++k) {
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        const int q = p0 + t;
                        const bool ok = unv[k] && !found[k] && q < lane_lim && q < deg[k];
                        cand[k][t] = ok ? __ldg(row[k] + q) : -1;
                        any = any || ok;
                    }
                }
                if (!any) break;
                uint32_t fw[W][CH];
#pragma unroll
                for (int k = 0; k < W; ++k)
#pragma unroll
                    for (int t = 0; t < CH; ++t)
                        fw[k][t] = cand[k][t] >= 0 ? ldro<CO>(front + (cand[k][t] >> 5)) : 0u;
#pragma unroll
                for (int k = 0; k < W; ++k) {
#pragma unroll
                    for (int t = 0; t < CH; ++t) {
                        if (!found[k] && cand[k][t] >= 0) {
                            ++ex[k];
                            if ((fw[k][t] >> (cand[k][t] & 31)) & 1u) {
                                found[k] = true;
                                p[k] = cand[k][t];
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < W; ++k) {
                unsigned pend = __ballot_sync(0xffffffffu, unv[k] && !found[k] && lane_lim < deg[k]);
                while (pend) {
                    const int L = __ffs(pend) - 1;
                    pend &= pend - 1;
                    const int32_t *lrow = (const int32_t *)__shfl_sync(
                        0xffffffffu, (unsigned long long)row[k], L);
                    const int ld = __shfl_sync(0xffffffffu, deg[k], L);
                    bool hit_any = false;
                    for (int q0 = lane_lim; q0 < ld; q0 += 64) {
                        int32_t uu[2];
                        bool hit[2];
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            const int q = q0 + 32 * t + (int)lane;
                            uu[t] = q < ld ? __ldg(lrow + q) : -1;
                        }
#pragma unroll
                        for (int t = 0; t < 2; ++t)
                            hit[t] = uu[t] >= 0 && ((ldro<CO>(front + (uu[t] >> 5)) >> (uu[t] & 31)) & 1u);
                        const unsigned h0 = __ballot_sync(0xffffffffu, hit[0]);
                        const unsigned h1 = __ballot_sync(0xffffffffu, hit[1]);
                        if (h0 | h1) {
                            const int t = h0 ? 0 : 1;
                            const int first = __ffs(h0 ? h0 : h1) - 1;
                            const int32_t pu = __shfl_sync(0xffffffffu, t ? uu[1] : uu[0], first);
                            if ((int)lane == L) {
                                found[k] = true;
                                p[k] = pu;
                                ex[k] += (q0 - lane_lim) + 32 * t + first + 1;
                            }
                            hit_any = true;
                            break;
                        }
                    }
                    if (!hit_any && (int)lane == L) ex[k] += ld - lane_lim;
                }
            }
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const int64_t v = v_c + (j + k) * 32;
                const unsigned fm = __ballot_sync(0xffffffffu, found[k]);
                if (found[k]) {
                    parent[v] = p[k];
                    if (level) level[v] = new_level;
                    my_mf += deg[k];
                }
                my_ex += ex[k];
                if (lane == 0) {
                    next_c[j + k] = fm;
                    if (fm) vis_c[j + k] = vw[k] | fm;
                    my_nf += __popc(fm);
                }
            }
        }
    }
    block_add3(my_nf, my_mf, my_ex, slot_next + T_NF, slot_next + T_MF, slot_next + T_EXAM);
}

template <int W, int CH, bool HEAD>
__global__ void __launch_bounds__(kBlock, 4) bu_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
    const int2 *__restrict__ head, int64_t nw_pad,
    uint32_t *__restrict__ visited, const uint32_t *__restrict__ front,
    uint32_t *__restrict__ next_bm, int32_t *__restrict__ parent, int32_t *__restrict__ level,
    int32_t new_level, int probe, unsigned long long *slot_next, int64_t *zero_slot, int span,
    int hskip) {
    bu_phase<W, CH, HEAD, false>(off, idx, head, nw_pad, visited, front, next_bm, parent, level,
                                 new_level, probe, slot_next, zero_slot, span, hskip);
}


// Bitmap -> list of its set bits after XOR with `flip`: flip = ~0 lists the
// vertices still to find from the visited bitmap (degree-0 vertices and ids
// past n are set in visited and so never listed); flip = 0 lists the pend
// bits of the two-pass bottom-up step. Same block scan as b2q_kernel.
template <bool CO>
__device__ __forceinline__ void bits_list_phase(const uint32_t *__restrict__ vis, uint32_t flip,
                                                int64_t nw, int32_t *__restrict__ list,
                                                unsigned long long *count) {
    __shared__ int wtot[kBlock / 32];
    __shared__ unsigned long long base_s;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    for (int64_t t0 = (int64_t)blockIdx.x * kBlock * 4; t0 < nw; t0 += (int64_t)gridDim.x * kBlock * 4) {
        const int64_t w0 = t0 + threadIdx.x * 4;
        uint32_t words[4];
        int c = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            words[k] = (w0 + k < nw) ? ld<CO>(vis + w0 + k) ^ flip : 0u;
            c += __popc(words[k]);
        }
        int tot;
        const int excl = warp_exclusive_scan(c, &tot);
        if (lane == 31) wtot[w] = tot;
        __syncthreads();
        int before = 0, all = 0;
        for (int i = 0; i < kBlock / 32; ++i) {
            if (i < (int)w) before += wtot[i];
            all += wtot[i];
        }
        if (threadIdx.x == 0) base_s = all ? atomicAdd(count, (unsigned long long)all) : 0ull;
        __syncthreads();
        unsigned long long pos = base_s + before + excl;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t x = words[k];
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1;
                list[pos++] = (int32_t)((w0 + k) * 32 + b);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) bits_list_kernel(const uint32_t *__restrict__ vis,
                                                           uint32_t flip, int64_t nw,
                                                           int32_t *__restrict__ list,
                                                           unsigned long long *count) {
    bits_list_phase<false>(vis, flip, nw, list, count);
}


// Bottom-up step over a compacted list of the vertices still to find: one
// lane per vertex, so a sparse layer keeps every lane busy. Each lane tests
// the first entries of its row itself, then the warp scans the rest of its
// lanes' rows together (first frontier neighbour in CSR order, after the
// head record's probe when head is set); a found vertex sets its next and
// visited bits with atomicOr, since no warp owns its word here.
constexpr int kFlat = 2;  // 32-entry chunks per round of the warp's flat row scan

template <bool CO>
__device__ __forceinline__ void bu_list_phase(
    const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
    const int2 *__restrict__ head, int hskip,
    const int32_t *__restrict__ list, const unsigned long long *count,
    uint32_t *__restrict__ visited, const uint32_t *__restrict__ front,
    uint32_t *__restrict__ next_bm, int32_t *__restrict__ parent, int32_t *__restrict__ level,
    int32_t new_level, int probe, unsigned long long *slot_next, int64_t *zero_slot,
    int mf_left = 0) {
    // mf_left = 1 (after the compact hub sweep): T_MF receives the degree sum
    // of the listed vertices left unvisited instead of that of the found ones
    // positions [p_start, lim) are tested by the lane itself
    const int p_start = head ? hskip : 0;
    const int lim = head ? (probe > hskip ? probe : hskip) : probe;
    if (blockIdx.x == 0 && threadIdx.x < kFields) zero_slot[threadIdx.x] = 0;
    const int64_t cnt = (int64_t)ld<CO>(count);
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t my_nf = 0, my_mf = 0, my_ex = 0;
    // Without head records (the row scans of the two-pass step) a lane's
    // list entry is loaded two iterations ahead and its row bounds one
    // iteration ahead, so an iteration's dependent chain is only row entries
    // then frontier words.
    const bool ahead = head == nullptr;
    const int64_t wstride = tw * 32;
    int32_t v_n1 = 0, v_n2 = 0;
    int64_t b_n1 = 0, e_n1 = 0;
    if (ahead) {
        const int64_t i1 = gw * 32 + lane, i2 = i1 + wstride;
        if (i1 < cnt) {
            v_n1 = ld<CO>(list + i1);
            b_n1 = off[v_n1];
            e_n1 = off[v_n1 + 1];
        }
        if (i2 < cnt) v_n2 = ld<CO>(list + i2);
    }
    for (int64_t base = gw * 32; base < cnt; base += wstride) {
        const int64_t i = base + lane;
        const bool have = i < cnt;
        int32_t v = 0;
        const int32_t *row = idx;
        int deg = 0, ex = 0;
        bool found = false;
        int32_t p = -1;
        if (have && ahead) {
            v = v_n1;
            row = idx + b_n1;
            deg = (int)(e_n1 - b_n1);
            // move the window: bounds of the next entry, the entry after it
            if (i + wstride < cnt) {
                b_n1 = off[v_n2];
                e_n1 = off[v_n2 + 1];
            }
            v_n1 = v_n2;
            v_n2 = i + 2 * wstride < cnt ? ld<CO>(list + i + 2 * wstride) : 0;
        } else if (have) {
            v = ld<CO>(list + i);
            if (head) {
                const int2 h = __ldg(head + v);
                deg = h.y;
                if (h.x >= 0) {
                    ex = 1;
                    if ((ldro<CO>(front + (h.x >> 5)) >> (h.x & 31)) & 1u) {
                        found = true;
                        p = h.x;
                    }
                }
                if (!found && deg > hskip) row = idx + off[v];
            } else {
                const int64_t b = off[v];
                row = idx + b;
                deg = (int)(off[v + 1] - b);
            }
        }
        for (int p0 = p_start; p0 < lim; p0 += 4) {
            int32_t cand[4];
            bool any = false;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int q = p0 + t;
                const bool ok = have && !found && q < lim && q < deg;
                cand[t] = ok ? __ldg(row + q) : -1;
                any = any || ok;
            }
            if (!any) break;
            uint32_t fw[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) fw[t] = cand[t] >= 0 ? ldro<CO>(front + (cand[t] >> 5)) : 0u;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (!found && cand[t] >= 0) {
                    ++ex;
                    if ((fw[t] >> (cand[t] & 31)) & 1u) {
                        found = true;
                        p = cand[t];
                    }
                }
            }
        }
        // Rows longer than lim: the warp scans the rest of all its lanes'
        // rows as one sequence, kFlat x 32 entries per round whatever the
        // rows' lengths (a short remainder no longer takes a whole round of
        // dependent loads). A row leaves the sequence at its first frontier
        // neighbour; the entries after it in the same round are loaded but
        // not counted, so parent and examined counts are those of a scan in
        // CSR order.
        int rem = (have && !found && lim < deg) ? deg - lim : 0;
        // address of sequence position 0 of this lane's rest (rest entry j of
        // the round is at seq + 4 j, for j in [excl, excl + rem))
        unsigned long long seq = (unsigned long long)(row + lim);
        while (__any_sync(0xffffffffu, rem > 0)) {
            int tot;
            const int excl = warp_exclusive_scan(rem, &tot);
            const unsigned long long at = seq - 4ull * (unsigned)excl;
            int32_t uu[kFlat];
            unsigned hb[kFlat];
#pragma unroll
            for (int c = 0; c < kFlat; ++c) {
                const int j = 32 * c + (int)lane;
                // owner = the last lane whose exclusive prefix is <= j
                int o = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int e = __shfl_sync(0xffffffffu, excl, o + step);
                    if (e <= j) o += step;
                }
                const unsigned long long oat = __shfl_sync(0xffffffffu, at, o);
                uu[c] = j < tot ? __ldg(reinterpret_cast<const int32_t *>(oat + 4ull * (unsigned)j))
                                : -1;
            }
#pragma unroll
            for (int c = 0; c < kFlat; ++c)
                hb[c] = __ballot_sync(0xffffffffu, uu[c] >= 0 && ((ldro<CO>(front + (uu[c] >> 5)) >>
                                                                   (uu[c] & 31)) & 1u));
            // this lane's entries of the round: [excl, hi); the first hit among them
            const int hi = min(excl + rem, 32 * kFlat);
            int first = -1;
#pragma unroll
            for (int c = kFlat - 1; c >= 0; --c) {
                const int a = max(excl - 32 * c, 0), b = min(hi - 32 * c, 32);
                if (a < b) {
                    const unsigned m = hb[c] & (b == 32 ? ~0u : (1u << b) - 1u) & ~((1u << a) - 1u);
                    if (m) first = 32 * c + __ffs(m) - 1;
                }
            }
            int32_t pu = -1;
#pragma unroll
            for (int c = 0; c < kFlat; ++c) {
                const int32_t x = __shfl_sync(0xffffffffu, uu[c], first & 31);
                if (first >> 5 == c) pu = x;
            }
            if (rem > 0 && excl < 32 * kFlat) {
                if (first >= 0) {
                    found = true;
                    p = pu;
                    ex += (deg - rem - lim) + (first - excl) + 1;  // up to and including the hit
                    rem = 0;
                } else {
                    rem -= hi - excl;
                    seq += 4ull * (unsigned)(hi - excl);
                    if (rem == 0) ex += deg - lim;
                }
            }
        }
        if (found) {
            const uint32_t bit = 1u << (v & 31);
            parent[v] = p;
            if (level) level[v] = new_level;
            atomicOr(next_bm + (v >> 5), bit);
            atomicOr(visited + (v >> 5), bit);
            if (!mf_left) my_mf += deg;
            my_nf += 1;
        } else if (mf_left && have) {
            my_mf += deg;
        }
        my_ex += ex;
    }
    block_add3(my_nf, my_mf, my_ex, slot_next + T_NF, slot_next + T_MF, slot_next + T_EXAM);
}

// First pass of the two-pass bottom-up step (hub head records): every
// unvisited vertex tests only its hub against the frontier. A warp owns 8
// consecutive bitmap words per round (lane i = bit i of each), so it writes
// their next and pend words and ORs the found bits into visited without
// atomics or block barriers; the warps run independently and keep many head
// loads in flight. pend marks the vertices whose hub missed and whose row
// must be scanned (bits_list_phase then compacts them for bu_list_phase); a
// vertex of degree 1 is not marked, since its only neighbour is the hub (its
// one-entry scan is counted here). Every word below nw_pad is written, so
// next and pend need no clearing.
// With init_out (the first sweep of a traversal that skipped the -1 fill),
// every vertex below n not reached in an earlier layer gets its outputs
// here: the hit's values, else -1 (a later find overwrites them), so the
// warp's stores cover whole sectors wherever no earlier-reached vertex sits.
template <bool CO>
__device__ __forceinline__ void bu_hub_phase(
    const int2 *__restrict__ head, int64_t nw_pad, uint32_t *__restrict__ visited,
    const uint32_t *__restrict__ front, uint32_t *__restrict__ next_bm,
    uint32_t *__restrict__ pend, int32_t *__restrict__ parent, int32_t *__restrict__ level,
    int32_t new_level, unsigned long long *slot_next, int64_t *zero_slot, int init_out,
    const uint32_t *__restrict__ base, int64_t n, int32_t root) {
    constexpr int R = 8;
    static_assert(32 % R == 0, "a round's R words must not cross nw_pad (a multiple of 32)");
    if (blockIdx.x == 0 && threadIdx.x < kFields) zero_slot[threadIdx.x] = 0;
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int64_t my_nf = 0, my_mf = 0, my_ex = 0;
    for (int64_t w0 = gw * R; w0 < nw_pad; w0 += tw * R) {  // nw_pad is a multiple of 32
        uint32_t vw[R];
        int2 h[R];
        uint32_t fw[R];
#pragma unroll
        for (int k = 0; k < R; ++k) vw[k] = ld<CO>(visited + w0 + k);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const bool unv = !((vw[k] >> lane) & 1u);  // bits past n are set
            h[k] = unv ? __ldg(head + (w0 + k) * 32 + lane) : make_int2(-1, 0);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) fw[k] = h[k].x >= 0 ? ldro<CO>(front + (h[k].x >> 5)) : 0u;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int64_t v = (w0 + k) * 32 + lane;
            const bool probed = h[k].x >= 0;
            const bool found = probed && ((fw[k] >> (h[k].x & 31)) & 1u);
            my_ex += probed ? (found || h[k].y > 1 ? 1 : 2) : 0;
            // one store per array for the whole warp (see the streaming sweep)
            const bool minus = !found && init_out && v < n && v != root &&
                               !(((vw[k] & ~__ldg(base + w0 + k)) >> lane) & 1u);
            if (found || minus) {
                parent[v] = found ? h[k].x : -1;
                if (level) level[v] = found ? new_level : -1;
            }
            if (found) {
                my_mf += h[k].y;
                my_nf += 1;
            }
            const unsigned fb = __ballot_sync(0xffffffffu, found);
            const unsigned pb = __ballot_sync(0xffffffffu, probed && !found && h[k].y > 1);
            if (lane == 0) {
                next_bm[w0 + k] = fb;
                pend[w0 + k] = pb;
                if (fb) visited[w0 + k] = vw[k] | fb;
            }
        }
    }
    block_add4(my_nf, my_mf, my_ex, my_nf, slot_next + T_NF, slot_next + T_MF,
               slot_next + T_EXAM, slot_next + T_HUB);
}

__global__ void __launch_bounds__(kBlock, 4) bu_hub_kernel(
    const int2 *__restrict__ head, int64_t nw_pad, uint32_t *__restrict__ visited,
    const uint32_t *__restrict__ front, uint32_t *__restrict__ next_bm,
    uint32_t *__restrict__ pend, int32_t *__restrict__ parent, int32_t *__restrict__ level,
    int32_t new_level, unsigned long long *slot_next, int64_t *zero_slot, int init_out,
    const uint32_t *__restrict__ base, int64_t n, int32_t root) {
    bu_hub_phase<false>(head, nw_pad, visited, front, next_bm, pend, parent, level, new_level,
                        slot_next, zero_slot, init_out, base, n, root);
}

// ---------------------------------------------------------------------------
// First pass of the two-pass bottom-up step on the compact hub records
// (hubc, 4 bytes per degree >= 1 vertex; host loop). Same per-vertex test as
// bu_hub_phase (Sec. 5.1: filter the unvisited vertices, probe), but the
// sweep needs no degree: a hit only stores its parent and level, and the
// switch counter e_f of the layer (Sec. 4) is taken as e_u before the layer
// minus e_u after it, where e_u after = the degree sum of the vertices still
// unvisited: a degree-1 vertex whose hub missed (counted here, bit 31 of its
// record) plus the hub misses the row scan does not find (counted by
// bu_list_phase with mf_left). The rank of vertex v among the degree >= 1
// vertices is wrank[v / 32] + the degree >= 1 vertices before it in its word.
//
// bu_hubc_stream_kernel (dense sweeps): bulk copies (cp.async.bulk,
// completion counted in bytes on an mbarrier) stream each warp's tiles of 8
// bitmap words (256 vertices, at most 1 KB of records) with the tile's
// visited, base and rank words into the warp's shared-memory ring, S tiles
// ahead, so the lanes make only the frontier-bit loads (L2) and the stores.
// bu_hubc_kernel (sparse sweeps) gathers the records of the unvisited
// vertices itself, 8 words per warp round.
// ---------------------------------------------------------------------------
constexpr unsigned long long kHubWaitNs = 1000000000ull;  // 1 s per bounded wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
// Makes the initialised barriers visible to the async proxy (the copy engine).
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Global -> shared bulk copy; both addresses 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the given phase parity: false once timeout_ns has passed.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity,
                                          unsigned long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > timeout_ns) return false;
    return true;
}

// L2 eviction policies (createpolicy): data streamed once through L2 is
// marked evict-first, the L2-resident frontier bitmap evict-last, so a sweep
// that moves a gigabyte through L2 does not push out the bitmap whose words
// every probe reads.
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint32_t ld_hint(const uint32_t *p, uint64_t pol) {
    uint32_t v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, unsigned bytes,
                                              uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

// Streaming sweep, one pipeline per warp: a warp owns tiles of kWarpTile
// bitmap words (256 vertices) and keeps S of them in flight in its own
// shared-memory ring, filled by bulk copies its lane 0 issues (the tile's
// compact records, its visited words and its {base, rank} words), each
// stage completing on its own mbarrier. No block-wide barrier: a warp
// waits only for its own copies and its own frontier loads.
constexpr int kWarpTile = 8;  // bitmap words per warp tile (a multiple of 4, dividing 32)
constexpr unsigned kWarpRecBytes = (kWarpTile * 32 + 8) * 4;  // records, 16-byte rounded
constexpr unsigned kWarpStageBytes = kWarpRecBytes + kWarpTile * 4 + kWarpTile * 8;
static_assert(kWarpStageBytes % 16 == 0, "stages keep bulk-copy destinations 16-byte aligned");
static_assert(kWarpTile % 4 == 0 && 32 % kWarpTile == 0, "tiles of 16-byte word groups that "
              "never cross nw_pad (a multiple of 32)");

// Predicated global accesses written as one predicated instruction each. The
// predicate is a word that is nonzero where the access happens, made by bit
// operations on the bitmap words, so no boolean is turned back into a word.
__device__ __forceinline__ uint32_t ld_hint_nz(const uint32_t *p, uint64_t pol, uint32_t u) {
    uint32_t v;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\tmov.b32 %0, 0;\n\t"
        "@q ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;\n\t}"
        : "=r"(v)
        : "l"(p), "l"(pol), "r"(u));
    return v;
}
__device__ __forceinline__ void st_cs_nz(int32_t *p, int32_t v, uint32_t u) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q st.global.cs.b32 [%0], %1;\n\t}"
                 ::"l"(p), "r"(v), "r"(u)
                 : "memory");
}
// Both stores under one predicate (parent and level of the same vertex).
__device__ __forceinline__ void st2_cs_nz(int32_t *p1, int32_t v1, int32_t *p2, int32_t v2,
                                          uint32_t u) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t"
                 "@q st.global.cs.b32 [%0], %1;\n\t@q st.global.cs.b32 [%2], %3;\n\t}"
                 ::"l"(p1), "r"(v1), "l"(p2), "r"(v2), "r"(u)
                 : "memory");
}

template <int S>
constexpr size_t hub_stream_smem() {
    return (size_t)(kBlock / 32) * ((size_t)S * kWarpStageBytes + (size_t)S * 16);
}

template <int S, bool INIT>
__global__ void __launch_bounds__(kBlock, 3) bu_hubc_stream_kernel(
    const uint32_t *__restrict__ hubc, const uint32_t *__restrict__ wrank,
    const uint2 *__restrict__ wmeta, int64_t nw_pad, uint32_t *__restrict__ visited,
    const uint32_t *__restrict__ front, uint32_t *__restrict__ next_bm,
    uint32_t *__restrict__ pend, int32_t *__restrict__ parent, int32_t *__restrict__ level,
    int32_t new_level, unsigned long long *slot_next, int64_t *zero_slot, int64_t n,
    int32_t root) {
    extern __shared__ __align__(128) unsigned char hub_smem[];
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    unsigned char *mine = hub_smem + (size_t)warp * ((size_t)S * kWarpStageBytes + (size_t)S * 16);
    uint64_t *full = reinterpret_cast<uint64_t *>(mine + (size_t)S * kWarpStageBytes);  // [S]
    uint32_t *rec0 = reinterpret_cast<uint32_t *>(full + S);                            // [S]
    if (blockIdx.x == 0 && threadIdx.x < kFields) zero_slot[threadIdx.x] = 0;
    const int64_t tiles = nw_pad / kWarpTile;  // nw_pad is a multiple of 32
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
    auto stage = [&](int s) { return mine + (size_t)s * kWarpStageBytes; };
    // lane 0: fill stage s with tile t, whose records are [r0, r1)
    auto issue = [&](int64_t t, int s, uint32_t r0, uint32_t r1) {
        const uint32_t a0 = r0 & ~3u, a1 = (r1 + 3u) & ~3u;  // hubc has spare records
        const unsigned rec_bytes = (a1 - a0) * 4u;
        rec0[s] = a0;
        mbar_expect_tx(full + s, rec_bytes + kWarpTile * 12);
        unsigned char *st = stage(s);
        if (rec_bytes) bulk_g2s_hint(st, hubc + a0, rec_bytes, full + s, pol_stream);
        bulk_g2s(st + kWarpRecBytes, visited + t * kWarpTile, kWarpTile * 4, full + s);
        bulk_g2s(st + kWarpRecBytes + kWarpTile * 4, wmeta + t * kWarpTile, kWarpTile * 8,
                 full + s);
    };
    uint32_t nr0 = 0, nr1 = 0;  // lane 0: record range of the next tile to issue
    if (lane == 0) {
        for (int s = 0; s < S; ++s) mbar_init(full + s, 1);
        mbar_init_fence();
        for (int s = 0; s < S; ++s) {
            const int64_t t = gw + (int64_t)s * tw;
            if (t < tiles) issue(t, s, wrank[t * kWarpTile], wrank[t * kWarpTile + kWarpTile]);
        }
        const int64_t t = gw + (int64_t)S * tw;
        if (t < tiles) {
            nr0 = wrank[t * kWarpTile];
            nr1 = wrank[t * kWarpTile + kWarpTile];
        }
    }
    __syncwarp();
    uint32_t c_nf = 0, c_d1 = 0, c_pr = 0;  // found, degree-1 misses, probed
    for (int64_t i = 0;; ++i) {
        const int64_t t = gw + i * tw;
        if (t >= tiles) break;
        const int s = (int)(i % S);
        const bool ok = mbar_wait(full + s, (unsigned)((i / S) & 1), kHubWaitNs);
        if (__any_sync(0xffffffffu, !ok)) {
            // a copy never completed: flag it, let this warp's copies in
            // flight land (bounded) and stop
            if (lane == 0) {
                atomicExch(reinterpret_cast<unsigned long long *>(slot_next + T_ERR), 1ull);
                for (int j = 0; j < S; ++j)
                    if (gw + (i + j) * tw < tiles)
                        mbar_wait(full + (int)((i + j) % S), (unsigned)(((i + j) / S) & 1),
                                  kHubWaitNs);
            }
            break;
        }
        const unsigned char *st = stage(s);
        const uint32_t *rec = reinterpret_cast<const uint32_t *>(st);
        const uint32_t *tv = reinterpret_cast<const uint32_t *>(st + kWarpRecBytes);
        const uint2 *tm = reinterpret_cast<const uint2 *>(st + kWarpRecBytes + kWarpTile * 4);
        const uint32_t a0 = rec0[s];
        const unsigned lt = lanemask_lt();
        uint32_t vw[kWarpTile], bw[kWarpTile], h[kWarpTile], fw[kWarpTile];
        const uint32_t bit = 1u << lane;
#pragma unroll
        for (int k = 0; k < kWarpTile; ++k) {
            vw[k] = tv[k];
            const uint2 m = tm[k];  // {base word, rank of the word's first vertex}
            bw[k] = m.x;
            // the index stays inside the stage's records for every lane (the
            // rank of the next degree >= 1 vertex), so the load needs no guard
            h[k] = rec[m.y - a0 + __popc(~m.x & lt)];
            // fw stays 0 where the lane is visited (unvisited implies degree >= 1)
            fw[k] = ld_hint_nz(front + ((h[k] & 0x7fffffffu) >> 5), pol_keep, ~vw[k] & bit);
        }
        uint32_t fbw[kWarpTile], d1w[kWarpTile];
        const int64_t vbase = t * (kWarpTile * 32);
        int32_t *const par_t = parent + vbase + lane;
        // level null: levels are written after the traversal (level pass)
        const bool lev_on = level != nullptr;
        int32_t *const lev_t = (lev_on ? level : parent) + vbase + lane;  // stores need lev_on
        if constexpr (INIT) {
            // A vertex not reached before is unvisited or of degree 0 (set in
            // both the visited and the base word) and gets -1 outputs, except
            // the ids past n (set in both as well) and a root of degree 0. In
            // the one or two tiles that hold those, they leave the tile's base
            // words here, so they count as reached and get no store.
            if (vbase + kWarpTile * 32 > n ||
                (uint64_t)((int64_t)root - vbase) < (uint64_t)(kWarpTile * 32)) {
#pragma unroll
                for (int k = 0; k < kWarpTile; ++k) {
                    const int64_t v = vbase + k * 32 + lane;
                    bw[k] &= ~__ballot_sync(0xffffffffu, v >= n || v == (int64_t)root);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kWarpTile; ++k) {
            // fw is 0 where the lane is visited: a set bit is a probed hit
            const uint32_t fbit = (fw[k] >> (h[k] & 31u)) & 1u;
            const bool found = fbit != 0u;
            const int32_t hub = (int32_t)(h[k] & 0x7fffffffu);
            fbw[k] = __ballot_sync(0xffffffffu, found);
            d1w[k] = __ballot_sync(0xffffffffu, (int32_t)h[k] < 0);  // degree 1 (where probed)
            if constexpr (INIT) {
                // one store per array for the whole warp (a hit's values,
                // else the -1 of a vertex not reached before): whole sectors
                const uint32_t out = ~(vw[k] & ~bw[k]) & bit;
                if (lev_on)
                    st2_cs_nz(par_t + k * 32, found ? hub : -1, lev_t + k * 32,
                              found ? new_level : -1, out);
                else
                    st_cs_nz(par_t + k * 32, found ? hub : -1, out);
            } else {
                if (lev_on)
                    st2_cs_nz(par_t + k * 32, hub, lev_t + k * 32, new_level, fbit);
                else
                    st_cs_nz(par_t + k * 32, hub, fbit);
            }
        }
        if (lane == 0) {
            uint32_t pbw[kWarpTile];
#pragma unroll
            for (int k = 0; k < kWarpTile; ++k) {
                const uint32_t miss = ~vw[k] & ~fbw[k];  // probed, hub not in the frontier
                pbw[k] = miss & ~d1w[k];                 // rows still to scan
                c_nf += __popc(fbw[k]);
                c_pr += __popc(~vw[k]);
                c_d1 += __popc(miss & d1w[k]);           // degree-1 misses: left unvisited
            }
            uint4 *nx = reinterpret_cast<uint4 *>(next_bm + t * kWarpTile);
            uint4 *pd = reinterpret_cast<uint4 *>(pend + t * kWarpTile);
            uint4 *vs = reinterpret_cast<uint4 *>(visited + t * kWarpTile);
#pragma unroll
            for (int q = 0; q < kWarpTile / 4; ++q) {
                const int k = 4 * q;
                nx[q] = make_uint4(fbw[k], fbw[k + 1], fbw[k + 2], fbw[k + 3]);
                pd[q] = make_uint4(pbw[k], pbw[k + 1], pbw[k + 2], pbw[k + 3]);
                vs[q] = make_uint4(vw[k] | fbw[k], vw[k + 1] | fbw[k + 1], vw[k + 2] | fbw[k + 2],
                                   vw[k + 3] | fbw[k + 3]);
            }
        }
        __syncwarp();  // the warp is done with stage s
        if (lane == 0) {
            const int64_t t2 = t + (int64_t)S * tw;
            if (t2 < tiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(t2, s, nr0, nr1);
                const int64_t t3 = t2 + tw;
                if (t3 < tiles) {
                    nr0 = wrank[t3 * kWarpTile];
                    nr1 = wrank[t3 * kWarpTile + kWarpTile];
                }
            }
        }
    }
    // the counts are held by lane 0
    const int64_t nf = lane == 0 ? c_nf : 0, d1 = lane == 0 ? c_d1 : 0,
                  pr = lane == 0 ? c_pr : 0;
    block_add4(nf, d1, pr + d1, nf, slot_next + T_NF, slot_next + T_MF, slot_next + T_EXAM,
               slot_next + T_HUB);
}

// Per-vertex step of the compact gather sweep for word w (visited word vw,
// base word bw) and the lane's record h (valid when the lane is unvisited).
__device__ __forceinline__ void hubc_word(
    int64_t w, uint32_t vw, uint32_t bw, uint32_t h, uint32_t fw, unsigned lane,
    uint32_t *__restrict__ visited, uint32_t *__restrict__ next_bm, uint32_t *__restrict__ pend,
    int32_t *__restrict__ parent, int32_t *__restrict__ level, int32_t new_level, int init_out,
    int64_t n, int32_t root, int64_t &my_nf, int64_t &my_left, int64_t &my_ex) {
    const int64_t v = w * 32 + lane;
    const bool probed = !((vw >> lane) & 1u);  // unvisited implies degree >= 1
    const int32_t hub = (int32_t)(h & 0x7fffffffu);
    const bool deg1 = (h >> 31) != 0u;
    const bool found = probed && ((fw >> (hub & 31)) & 1u);
    my_ex += probed ? (found || !deg1 ? 1 : 2) : 0;
    my_left += (probed && !found && deg1) ? 1 : 0;
    my_nf += found ? 1 : 0;
    // one store per array for the whole warp (whole sectors)
    const bool minus = !found && init_out && v < n && v != root && !(((vw & ~bw) >> lane) & 1u);
    if (found || minus) {
        __stcs(parent + v, found ? hub : -1);
        if (level) __stcs(level + v, found ? new_level : -1);
    }
    const unsigned fb = __ballot_sync(0xffffffffu, found);
    const unsigned pb = __ballot_sync(0xffffffffu, probed && !found && !deg1);
    if (lane == 0) {
        next_bm[w] = fb;
        pend[w] = pb;
        if (fb) visited[w] = vw | fb;
    }
}

// Sparse sweeps: the warp gathers the records of its unvisited vertices,
// 8 words per round (lane i = bit i of each).
__global__ void __launch_bounds__(kBlock, 4) bu_hubc_kernel(
    const uint32_t *__restrict__ hubc, const uint32_t *__restrict__ wrank, int64_t nw_pad,
    uint32_t *__restrict__ visited, const uint32_t *__restrict__ front,
    uint32_t *__restrict__ next_bm, uint32_t *__restrict__ pend, int32_t *__restrict__ parent,
    int32_t *__restrict__ level, int32_t new_level, unsigned long long *slot_next,
    int64_t *zero_slot, int init_out, const uint32_t *__restrict__ base, int64_t n,
    int32_t root) {
    constexpr int R = 8;
    static_assert(32 % R == 0, "a round's R words must not cross nw_pad (a multiple of 32)");
    if (blockIdx.x == 0 && threadIdx.x < kFields) zero_slot[threadIdx.x] = 0;
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t pol_stream = l2_evict_first(), pol_keep = l2_evict_last();
    int64_t my_nf = 0, my_left = 0, my_ex = 0;
    for (int64_t w0 = gw * R; w0 < nw_pad; w0 += tw * R) {
        uint32_t vw[R], bw[R], h[R], fw[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            vw[k] = visited[w0 + k];
            bw[k] = __ldg(base + w0 + k);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const bool probed = !((vw[k] >> lane) & 1u);
            h[k] = probed ? ld_hint(hubc + __ldg(wrank + w0 + k) + __popc(~bw[k] & lanemask_lt()),
                                    pol_stream)
                          : 0u;
        }
#pragma unroll
        for (int k = 0; k < R; ++k)
            fw[k] = !((vw[k] >> lane) & 1u) ? ld_hint(front + ((h[k] & 0x7fffffffu) >> 5), pol_keep)
                                            : 0u;
#pragma unroll
        for (int k = 0; k < R; ++k)
            hubc_word(w0 + k, vw[k], bw[k], h[k], fw[k], lane, visited, next_bm, pend, parent,
                      level, new_level, init_out, n, root, my_nf, my_left, my_ex);
    }
    block_add4(my_nf, my_left, my_ex, my_nf, slot_next + T_NF, slot_next + T_MF,
               slot_next + T_EXAM, slot_next + T_HUB);
}

__global__ void __launch_bounds__(kBlock) bu_list_kernel(
    const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
    const int2 *__restrict__ head, int hskip,
    const int32_t *__restrict__ list, const unsigned long long *count,
    uint32_t *__restrict__ visited, const uint32_t *__restrict__ front,
    uint32_t *__restrict__ next_bm, int32_t *__restrict__ parent, int32_t *__restrict__ level,
    int32_t new_level, int probe, unsigned long long *slot_next, int64_t *zero_slot,
    int mf_left) {
    bu_list_phase<false>(off, idx, head, hskip, list, count, visited, front, next_bm, parent,
                         level, new_level, probe, slot_next, zero_slot, mf_left);
}


__global__ void count_bits_kernel(const uint32_t *__restrict__ bits, int64_t nw,
                                  unsigned long long *count) {
    int64_t c = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += stride)
        c += __popc(bits[w]);
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, (unsigned long long)c);
}

constexpr auto BU1 = bu_kernel<1, 4, false>;
constexpr auto BU2 = bu_kernel<2, 4, false>;
constexpr auto BU4 = bu_kernel<4, 2, false>;
constexpr auto BU1H = bu_kernel<1, 4, true>;
constexpr auto BU2H = bu_kernel<2, 4, true>;
constexpr auto BU4H = bu_kernel<4, 2, true>;

// Frontier bitmap -> queue: each thread takes 4 consecutive words, a block
// scan orders the set bits, one atomicAdd per block reserves queue space.
template <bool CO>
__device__ __forceinline__ void b2q_phase(const uint32_t *__restrict__ bm, int64_t nw,
                                                     int32_t *__restrict__ q,
                                                     unsigned long long *count) {
    __shared__ int wtot[kBlock / 32];
    __shared__ unsigned long long base_s;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    for (int64_t t0 = (int64_t)blockIdx.x * kBlock * 4; t0 < nw; t0 += (int64_t)gridDim.x * kBlock * 4) {
        const int64_t w0 = t0 + threadIdx.x * 4;
        uint32_t words[4];
        int c = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            words[k] = (w0 + k < nw) ? ld<CO>(bm + w0 + k) : 0u;
            c += __popc(words[k]);
        }
        int tot;
        int excl = warp_exclusive_scan(c, &tot);
        if (lane == 31) wtot[w] = tot;
        __syncthreads();
        int before = 0, all = 0;
        for (int i = 0; i < kBlock / 32; ++i) {
            if (i < (int)w) before += wtot[i];
            all += wtot[i];
        }
        if (threadIdx.x == 0) base_s = all ? atomicAdd(count, (unsigned long long)all) : 0ull;
        __syncthreads();
        unsigned long long pos = base_s + before + excl;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t x = words[k];
            while (x) {
                const int b = __ffs(x) - 1;
                x &= x - 1;
                q[pos++] = (int32_t)((w0 + k) * 32 + b);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBlock) b2q_kernel(const uint32_t *__restrict__ bm, int64_t nw,
                                                     int32_t *__restrict__ q,
                                                     unsigned long long *count) {
    b2q_phase<false>(bm, nw, q, count);
}


__global__ void validate_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ idx,
                                int64_t n, int64_t nnz, int *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t0 == 0 && (off[0] != 0 || off[n] != nnz)) *bad = 1;
    for (int64_t v = t0; v < n; v += stride)
        if (off[v] > off[v + 1]) *bad = 1;
    for (int64_t e = t0; e < nnz; e += stride)
        if (idx[e] < 0 || idx[e] >= n) *bad = 1;
}

// Row-order and symmetry check (BFS_VALIDATE_SYMMETRIC), run only once the
// offsets and indices passed validate_kernel: a warp per row; each entry u of
// row v must exceed its predecessor and have v in row u (binary search).
__global__ void symmetric_kernel(const int64_t *__restrict__ off,
                                 const int32_t *__restrict__ idx, int64_t n, int *bad) {
    const unsigned lane = lane_id();
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t tw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = gw; v < n; v += tw) {
        const int64_t b = off[v], e = off[v + 1];
        bool ok = true;
        for (int64_t q = b + lane; q < e; q += 32) {
            const int32_t u = idx[q];
            if (q > b && idx[q - 1] >= u) ok = false;
            int64_t lo = off[u], hi = off[u + 1];
            while (lo < hi) {
                const int64_t mid = lo + ((hi - lo) >> 1);
                if (idx[mid] < v) lo = mid + 1;
                else hi = mid;
            }
            if (lo == off[u + 1] || idx[lo] != v) ok = false;
        }
        if (!ok) atomicExch(bad, 1);
    }
}

bool config_ok(const bfs_config &c) {
    if (c.policy < 0 || c.policy > 2) return false;
    if (c.policy == BFS_POLICY_FORCED && (c.forced_len < 1 || c.forced_len > 64)) return false;
    if (!(c.alpha > 0) || !(c.beta > 0)) return false;
    if (c.bu_probe < 1 || c.bu_probe > 64) return false;
    if (c.td_warp_degree < 1 || c.td_grid_degree < c.td_warp_degree) return false;
    if (c.bu_words != 1 && c.bu_words != 2 && c.bu_words != 4) return false;
    if (c.td_claim != 0 && c.td_claim != 1) return false;
    if (c.bu_head < 0 || c.bu_head > 2) return false;
    if (c.host_async != 0 && c.host_async != 1) return false;
    if (c.parent_min != 0 && c.parent_min != 1) return false;
    if (c.prune_components != 0 && c.prune_components != 1) return false;
    if (c.bu_list_percent < 0 || c.bu_list_percent > 100) return false;
    if (c.device_loop < 0 || c.device_loop > 4) return false;
    if (c.timing < 0 || c.timing > 2) return false;
    if (c.hub_stream_stages != 0 && c.hub_stream_stages != 2 && c.hub_stream_stages != 3 &&
        c.hub_stream_stages != 4 && c.hub_stream_stages != 6 && c.hub_stream_stages != 8)
        return false;
    if (c.hub_stream_percent < 0 || c.hub_stream_percent > 100) return false;
    if (c.level_pass != 0 && c.level_pass != 1) return false;
    return true;
}

// The streaming hub sweep for a stage count, its dynamic shared memory, and
// its resident blocks per SM (queried once per graph and stage count; the
// shared-memory limit is raised where a count needs more than the default).
using HubStreamFn = void (*)(const uint32_t *, const uint32_t *, const uint2 *, int64_t,
                             uint32_t *, const uint32_t *, uint32_t *, uint32_t *, int32_t *,
                             int32_t *, int32_t, unsigned long long *, int64_t *, int64_t,
                             int32_t);
// init: the sweep also writes the -1 of every vertex not reached before it
HubStreamFn hub_stream_fn(int stages, bool init) {
    switch (stages) {
        case 2: return init ? bu_hubc_stream_kernel<2, true> : bu_hubc_stream_kernel<2, false>;
        case 3: return init ? bu_hubc_stream_kernel<3, true> : bu_hubc_stream_kernel<3, false>;
        case 4: return init ? bu_hubc_stream_kernel<4, true> : bu_hubc_stream_kernel<4, false>;
        case 6: return init ? bu_hubc_stream_kernel<6, true> : bu_hubc_stream_kernel<6, false>;
        default: return init ? bu_hubc_stream_kernel<8, true> : bu_hubc_stream_kernel<8, false>;
    }
}
size_t hub_stream_smem_bytes(int stages) {
    switch (stages) {
        case 2: return hub_stream_smem<2>();
        case 3: return hub_stream_smem<3>();
        case 4: return hub_stream_smem<4>();
        case 6: return hub_stream_smem<6>();
        default: return hub_stream_smem<8>();
    }
}

// Alg. 3 switch, read as hysteresis (Table 2 layer 5 rules out the
// state-free reading). Returns 1 for bottom-up.
__host__ __device__ int decide(const bfs_config &c, int cur_bu, int d, int64_t n, int64_t n_f,
                               int64_t m_f, int64_t n_u, int64_t m_u) {
    if (c.policy == BFS_POLICY_FORCED)
        return c.forced[d < c.forced_len - 1 ? d : c.forced_len - 1] ? 1 : 0;
    if (c.policy == BFS_POLICY_VERTEX) {
        if (!cur_bu) return n_f > (n_u >> 10) ? 1 : 0;
        return n_f < (n >> 6) ? 0 : 1;
    }
    if (!cur_bu) return ((double)m_f > (double)m_u / c.alpha) ? 1 : 0;
    return ((double)n_f < (double)n / c.beta) ? 0 : 1;
}


// ---------------------------------------------------------------------------
// Device-side layer loop (cfg.device_loop): the traversal of bfs_run in one
// cooperative launch. Every block runs the same loop over layers, reads the
// layer counters after a grid barrier and so takes the same Alg. 3 decision
// and the same launch parameters the host loop would compute; the phases are
// the host loop's kernels as device functions, with coherent (L2) loads for
// data other blocks wrote earlier in the launch.
// ---------------------------------------------------------------------------
constexpr int kSsMaxRecords = 4096;  // per-layer records kept for statistics

// Words per dense bottom-up warp task: 32 (a whole chunk) unless that leaves
// fewer than two tasks per warp, then halved down to the words in flight.
__host__ __device__ inline int bu_span(int64_t nchunks, int w, int64_t warps) {
    int span = 32;
    while (span > w && nchunks * (32 / span) < 2 * warps) span >>= 1;
    return span;
}

struct SsPersist {
    const int64_t *off;
    const int32_t *idx;
    const int2 *head;  // head records for the bottom-up probe, or null
    int hskip;
    uint32_t *pend;    // two-pass bottom-up (hub records): hub misses, else null
    int64_t n, nnz, nw, nw_pad, deg0;
    uint32_t *visited, *bm_a, *bm_b;
    int32_t *q_a, *q_b, *big;
    int32_t *parent, *level;
    int64_t *trace;    // ring of kRing slots; slot 0 written by init_kernel
    int64_t *layers;   // [kSsMaxRecords][8] per-layer record
    int64_t *result;   // [0] layers, [1] status, [2] degree sum over frontiers
    unsigned *bar;     // barrier count, generation
    int32_t *err;
    bfs_config cfg;
    unsigned long long timeout_ns;
    // start state (layer, Alg. 3 counters, direction, queue) and whether to
    // stop at the first bottom-up decision: the hybrid loop runs stretches
    // of top-down layers here and the bottom-up layers from the host
    int64_t d0, n_f0, m_f0, n_u0, m_u0, degsum0;
    int cur_bu0, have_queue0, stop_at_bu;
};

__global__ void __launch_bounds__(kBlock, 4) bfs_persistent_kernel(SsPersist p) {
    const unsigned expected = gridDim.x;
    const int64_t td_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // m_f0 < 0: a whole traversal from the root (its degree is in slot 0)
    int64_t n_f = p.n_f0, m_f = p.m_f0 < 0 ? __ldcg(p.trace + T_MF) : p.m_f0;
    int64_t n_u = p.n_u0, m_u = p.m_f0 < 0 ? p.nnz - m_f : p.m_u0, degsum = p.degsum0;
    int cur_bu = p.cur_bu0, status = BFS_OK;
    int d = (int)p.d0;
    bool have_queue = p.have_queue0 != 0;
    for (; n_f > 0; ++d) {
        if (d > p.n) {  // a BFS has at most n layers: the counters are inconsistent
            status = BFS_ERR_INTERNAL;
            break;
        }
        const int next_bu = decide(p.cfg, cur_bu, d, p.n, n_f, m_f, n_u, m_u);
        if (p.stop_at_bu && next_bu) break;  // the host runs the bottom-up layer
        cur_bu = next_bu;
        degsum += m_f;
        int64_t *sc = p.trace + (d % kRing) * kFields;
        int64_t *sn = p.trace + ((d + 1) % kRing) * kFields;
        int64_t *sz = p.trace + ((d + 2) % kRing) * kFields;
        uint32_t *front = (d & 1) ? p.bm_b : p.bm_a;
        uint32_t *next = (d & 1) ? p.bm_a : p.bm_b;
        int32_t *q_cur = (d & 1) ? p.q_b : p.q_a;
        int32_t *q_next = (d & 1) ? p.q_a : p.q_b;
        int converted = 0;
        if (!cur_bu) {
            if (!have_queue) {
                b2q_phase<true>(front, p.nw, q_cur, (unsigned long long *)(sc + T_CONV));
                converted = 1;
            }
            for (int64_t i = t0; i < p.nw_pad; i += stride) next[i] = 0u;
            if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
                status = BFS_ERR_TIMEOUT;
                break;
            }
            const int queue_mode = m_f <= kQueueModeMaxEdges ? 1 : 0;
            const int defer = td_defer(queue_mode, n_u - p.deg0, p.nw);
            TdArgs a{p.off, p.idx, p.visited, next, p.parent, p.level, q_next,
                     (unsigned long long *)(sn + T_NF), d + 1, queue_mode, p.cfg.td_claim, defer};
            int64_t pw = (n_f + td_warps - 1) / td_warps;
            const int per_warp = (int)(pw < 1 ? 1 : (pw > 32 ? 32 : pw));
            int64_t gd = m_f / td_warps;
            if (gd < 4 * (int64_t)p.cfg.td_warp_degree) gd = 4 * (int64_t)p.cfg.td_warp_degree;
            if (gd > p.cfg.td_grid_degree) gd = p.cfg.td_grid_degree;
            td_phase<true>(a, q_cur, n_f, per_warp, p.big, (unsigned long long *)(sc + T_BIG),
                           (unsigned long long *)(sn + T_MF), p.cfg.td_warp_degree, gd, sz);
            if (m_f >= gd) {
                if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
                    status = BFS_ERR_TIMEOUT;
                    break;
                }
                td_big_phase<true>(a, p.big, (const unsigned long long *)(sc + T_BIG),
                                   (unsigned long long *)(sn + T_MF));
            }
            if (defer) {
                if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
                    status = BFS_ERR_TIMEOUT;
                    break;
                }
                td_post_phase<true>(p.off, next, p.nw, p.level, d + 1,
                                    (unsigned long long *)(sn + T_NF),
                                    (unsigned long long *)(sn + T_MF));
            }
            have_queue = queue_mode != 0;
        } else {
            const int64_t active = n_u - p.deg0;
            if (p.cfg.bu_list_percent > 0 && active * 100 <= (int64_t)p.cfg.bu_list_percent * p.n) {
                for (int64_t i = t0; i < p.nw_pad; i += stride) next[i] = 0u;
                bits_list_phase<true>(p.visited, ~0u, p.nw, q_next,
                                           (unsigned long long *)(sc + T_ULIST));
                if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
                    status = BFS_ERR_TIMEOUT;
                    break;
                }
                bu_list_phase<true>(p.off, p.idx, p.head, p.hskip, q_next,
                                    (const unsigned long long *)(sc + T_ULIST),
                                    p.visited, front, next, p.parent, p.level, d + 1,
                                    p.cfg.bu_probe, (unsigned long long *)sn, sz);
                converted = 2;
            } else if (p.pend && p.nw >= 8 * td_warps) {
                // two passes: hub probes over the words, then the rows of the
                // vertices whose hub missed, one lane each
                bu_hub_phase<true>(p.head, p.nw_pad, p.visited, front, next, p.pend, p.parent,
                                   p.level, d + 1, (unsigned long long *)sn, sz, 0, nullptr, p.n,
                                   -1);
                if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
                    status = BFS_ERR_TIMEOUT;
                    break;
                }
                bits_list_phase<true>(p.pend, 0u, p.nw, q_next, (unsigned long long *)(sc + T_ULIST));
                if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
                    status = BFS_ERR_TIMEOUT;
                    break;
                }
                bu_list_phase<true>(p.off, p.idx, nullptr, 0, q_next,
                                    (const unsigned long long *)(sc + T_ULIST), p.visited, front,
                                    next, p.parent, p.level, d + 1, p.cfg.bu_probe,
                                    (unsigned long long *)sn, sz);
                converted = 3;
            } else {
                if (p.head)
                    bu_phase<2, 4, true, true>(p.off, p.idx, p.head, p.nw_pad, p.visited, front,
                                               next, p.parent, p.level, d + 1, p.cfg.bu_probe,
                                               (unsigned long long *)sn, sz,
                                               bu_span(p.nw_pad >> 5, 2, td_warps), p.hskip);
                else
                    bu_phase<4, 2, false, true>(p.off, p.idx, nullptr, p.nw_pad, p.visited, front,
                                                next, p.parent, p.level, d + 1, p.cfg.bu_probe,
                                                (unsigned long long *)sn, sz,
                                                bu_span(p.nw_pad >> 5, 4, td_warps), 0);
            }
            have_queue = false;
        }
        if (!grid_barrier(p.bar, p.err, expected, p.timeout_ns)) {
            status = BFS_ERR_TIMEOUT;
            break;
        }
        const int64_t found = __ldcg(sn + T_NF), m_new = __ldcg(sn + T_MF);
        if (blockIdx.x == 0 && threadIdx.x == 0 && d < kSsMaxRecords) {
            int64_t *rec = p.layers + (int64_t)d * 8;
            rec[0] = cur_bu;
            rec[1] = converted;
            rec[2] = n_f;
            rec[3] = m_f;
            rec[4] = n_u;
            rec[5] = m_u;
            rec[6] = cur_bu ? __ldcg(sn + T_EXAM) : m_f;
            rec[7] = found;
        }
        n_u -= found;
        m_u -= m_new;
        n_f = found;
        m_f = m_new;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.result[0] = d;
        p.result[1] = status;
        p.result[2] = degsum;
        p.result[8] = n_f;
        p.result[9] = m_f;
        p.result[10] = n_u;
        p.result[11] = m_u;
        p.result[12] = have_queue ? 1 : 0;
        p.result[13] = cur_bu;
    }
}

// result header: [0] layers (or the layer the run stopped at), [1] status,
// [2] degree sum, [4..5] grid barrier and error word, [8..13] end state
constexpr int kPctlHead = 16;
constexpr size_t kPctlSsBytes = (size_t)kSsMaxRecords * 8 * 8 + kPctlHead * 8;
constexpr int64_t kDeviceLoopAutoMaxN = 1ll << 25;  // device_loop = 2: on up to this n

// State of the layer loop between layers, shared by the host loop and the
// persistent kernel's stretches of top-down layers.
struct LoopState {
    int64_t d = 0, n_f = 1, m_f = -1, n_u = 0, m_u = 0, degsum = 0;
    int cur_bu = 0, have_queue = 1;
};

// Runs layers from state `s` in one cooperative launch of
// bfs_persistent_kernel (init_kernel has already run on `st`), appends their
// records to g->last and leaves the end state in `s`. With stop_at_bu the
// launch returns at the first bottom-up decision (s.d is then that layer);
// otherwise it runs to the end of the traversal.
bfs_status run_device_segment(bfs_graph *g, int32_t *level, int32_t *parent, cudaStream_t st,
                              LoopState &s, bool stop_at_bu) {
    if (!g->pctl) {
        GB_CK(dev_malloc(&g->pctl, kPctlSsBytes));
        GB_CK(host_malloc(&g->h_pctl, kPctlSsBytes));
    }
    if (g->persist_blocks_per_sm <= 0) {
        GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->persist_blocks_per_sm,
                                                            bfs_persistent_kernel, kBlock, 0));
        if (g->persist_blocks_per_sm <= 0) {
            set_error("bfs_run: the device-loop kernel does not fit on an SM");
            return BFS_ERR_CUDA;
        }
    }
    // layout: the kPctlHead-word result header, then the per-layer records,
    // so one small copy covers short traversals
    int64_t *result = g->pctl;
    GB_CK(cudaMemsetAsync(result, 0, kPctlHead * 8, st));
    SsPersist p;
    p.off = g->off;
    p.idx = g->idx;
    p.n = g->n;
    p.nnz = g->nnz;
    p.nw = g->nw;
    p.nw_pad = g->nw_pad;
    p.deg0 = g->deg0;
    p.visited = g->visited;
    p.bm_a = g->bm_a;
    p.bm_b = g->bm_b;
    p.q_a = g->q_a;
    p.q_b = g->q_b;
    p.big = g->big;
    p.parent = parent;
    p.level = level;
    p.trace = g->trace;
    p.layers = g->pctl + kPctlHead;
    p.result = result;
    p.bar = (unsigned *)(result + 4);
    p.err = (int32_t *)(p.bar + 2);
    p.cfg = g->cfg;
    p.head = g->cfg.bu_head ? g->head : nullptr;
    p.hskip = g->cfg.bu_head == 1 ? 1 : 0;
    p.pend = g->cfg.bu_head == 2 ? g->pend : nullptr;
    p.timeout_ns = 2000000000ull;  // 2 s per barrier wait
    p.d0 = s.d;
    p.n_f0 = s.n_f;
    p.m_f0 = s.m_f;
    p.n_u0 = s.n_u;
    p.m_u0 = s.m_u;
    p.degsum0 = s.degsum;
    p.cur_bu0 = s.cur_bu;
    p.have_queue0 = s.have_queue;
    p.stop_at_bu = stop_at_bu ? 1 : 0;
    void *args[] = {&p};
    // Grid sized to the graph: barrier cost grows with the block count, and a
    // small graph cannot use the whole GPU anyway (one block per 2048
    // vertices, at least one per SM, at most the resident maximum).
    const int64_t full = (int64_t)g->persist_blocks_per_sm * sm_count();
    const int64_t want = std::max<int64_t>(sm_count(), (g->n + 2047) / 2048);
    const int grid = (int)std::min<int64_t>(full, want);
    GB_CK(cudaLaunchCooperativeKernel((const void *)bfs_persistent_kernel, dim3(grid), dim3(kBlock),
                                      args, 0, st));
    count_launch();
    constexpr int64_t kFirst = 64;  // records fetched with the result
    const int64_t first = std::min<int64_t>(s.d + kFirst, kSsMaxRecords);
    GB_CK(cudaMemcpyAsync(g->h_pctl, g->pctl, (size_t)(kPctlHead + first * 8) * 8,
                          cudaMemcpyDeviceToHost, st));
    GB_CK(cudaStreamSynchronize(st));
    const int64_t *hres = g->h_pctl;
    const int64_t end = hres[0];
    if (std::min<int64_t>(end, kSsMaxRecords) > first) {
        const int64_t more = std::min<int64_t>(end, kSsMaxRecords) - first;
        GB_CK(cudaMemcpyAsync(g->h_pctl + kPctlHead + first * 8, g->pctl + kPctlHead + first * 8,
                              (size_t)more * 64, cudaMemcpyDeviceToHost, st));
        GB_CK(cudaStreamSynchronize(st));
    }
    for (int64_t d = s.d; d < end && d < kSsMaxRecords; ++d) {
        const int64_t *rec = g->h_pctl + kPctlHead + d * 8;
        bfs_layer_stats ls;
        memset(&ls, 0, sizeof ls);
        ls.direction = (int32_t)rec[0];
        ls.converted = (int32_t)rec[1];
        ls.n_f = rec[2];
        ls.m_f = rec[3];
        ls.n_u = rec[4];
        ls.m_u = rec[5];
        ls.examined = rec[6];
        ls.found = rec[7];
        g->last.push_back(ls);
    }
    if (hres[1] == BFS_ERR_TIMEOUT) {
        set_error("bfs_run: a grid barrier wait of the device loop ran out");
        return BFS_ERR_TIMEOUT;
    }
    if (hres[1] != BFS_OK) {
        set_error("bfs_run: the device loop stopped (status %lld)", (long long)hres[1]);
        return (bfs_status)hres[1];
    }
    s.d = end;
    s.degsum = hres[2];
    s.n_f = hres[8];
    s.m_f = hres[9];
    s.n_u = hres[10];
    s.m_u = hres[11];
    s.have_queue = (int)hres[12];
    s.cur_bu = (int)hres[13];
    return BFS_OK;
}

// The whole traversal as one cooperative launch.
bfs_status run_device_loop(bfs_graph *g, int32_t *level, int32_t *parent, cudaStream_t st) {
    LoopState s;
    s.n_u = g->n - 1;  // m_f < 0: the kernel reads the root's degree
    const bfs_status r = run_device_segment(g, level, parent, st, s, false);
    g->last_component_edges = s.degsum / 2;
    return r;
}

// Graph loop (device_loop = 3): the layer loop as one CUDA graph whose
// control flow stays on the device. A WHILE node repeats {gl_step_kernel,
// SWITCH}: the step kernel closes the layer that just ran (its record and
// the Alg. 3 counters), applies the Alg. 3 switch for the next layer and
// picks that layer's variant, which the SWITCH node runs. The variants are
// the host loop's kernel sequences, as wrappers that read their per-layer
// arguments from the device-resident GlRun. There is no host round trip
// between layers; one launch runs at most kGlCap layers, so every launch
// ends, and the host launches again while the traversal is not done.
enum GlCase : unsigned {
    GL_TD = 0,         // top-down; + 1 queue rebuilt first, + 2 grid-spread vertices,
                       //           + 4 deferred level pass   (cases 0..7)
    GL_LIST = 8,       // sparse bottom-up layer over the list of unvisited vertices
    GL_LIST_FILL = 9,  //   the same after the -1 fill of the outputs
    GL_TWO = 10,       // two-pass bottom-up: hub sweep, list of misses, row scans
    GL_ONE = 11,       // one-pass bottom-up
    GL_ONE_FILL = 12,  //   the same after the -1 fill
    GL_CASES = 13      // a value >= GL_CASES runs no layer
};
constexpr int kGlCap = 256;  // layers per graph launch
constexpr int kGlRec = 10;   // int64 fields per layer record
constexpr size_t kGlRunBytes = 256;

struct GlRun {
    int64_t n_f, m_f, n_u, m_u, degsum, kernels, grid_deg;
    int64_t *sc, *sn, *sz;  // trace slots of the planned layer
    uint32_t *front, *next;
    int32_t *q_cur, *q_next;
    int32_t *level, *parent;
    int32_t d, cur_bu, have_queue, filled, status, done, pending, iter;
    int32_t root, converted, per_warp, queue_mode, defer, init_out;
};
static_assert(sizeof(GlRun) <= kGlRunBytes, "GlRun must fit its slot");

struct GlStatic {
    const int64_t *off;
    const int32_t *idx;
    const int2 *head;  // head records (bu_head != 0), else null
    int hskip;
    const uint32_t *base_vis;
    uint32_t *visited, *bm_a, *bm_b, *pend;
    int32_t *q_a, *q_b, *big;
    int64_t *trace;
    int64_t *rec;  // [kSsMaxRecords][kGlRec] per-layer records
    GlRun *run;
    int64_t n, nnz, nw, nw_pad, deg0, td_warps;
    int two_pass, bu_span_w;
    bfs_config cfg;
    cudaGraphConditionalHandle h_loop, h_case, h_fill;
};

__global__ void gl_start_kernel(GlStatic s, int32_t *level, int32_t *parent, int32_t root,
                                int filled) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    GlRun &r = *s.run;
    r.n_f = 1;
    r.m_f = s.trace[T_MF];  // degree of the root (init_kernel)
    r.n_u = s.n - 1;
    r.m_u = s.nnz - r.m_f;
    r.degsum = 0;
    r.kernels = 0;
    r.d = 0;
    r.cur_bu = 0;
    r.have_queue = 1;
    r.filled = filled;
    r.status = BFS_OK;
    r.done = 0;
    r.pending = 0;
    r.iter = 0;
    r.level = level;
    r.parent = parent;
    r.root = root;
}

__global__ void gl_begin_kernel(GlStatic s) {
    if (threadIdx.x == 0 && blockIdx.x == 0) s.run->iter = 0;
}

__global__ void gl_step_kernel(GlStatic s) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    GlRun &r = *s.run;
    r.kernels += 1;
    if (r.pending) {  // close the layer that just ran
        const int64_t found = r.sn[T_NF], m_new = r.sn[T_MF];
        if (r.d < kSsMaxRecords) {
            int64_t *rec = s.rec + (int64_t)r.d * kGlRec;
            rec[0] = r.cur_bu;
            rec[1] = r.converted;
            rec[2] = r.n_f;
            rec[3] = r.m_f;
            rec[4] = r.n_u;
            rec[5] = r.m_u;
            rec[6] = r.cur_bu ? r.sn[T_EXAM] : r.m_f;
            rec[7] = found;
            rec[8] = r.converted == 3 ? r.sn[T_HUB] : 0;
            rec[9] = 0;
        }
        r.n_u -= found;
        r.m_u -= m_new;
        r.n_f = found;
        r.m_f = m_new;
        r.have_queue = r.cur_bu ? 0 : r.queue_mode;
        r.d += 1;
        r.pending = 0;
    }
    bool go = r.status == BFS_OK && r.n_f > 0;
    if (go && r.d > s.n) {  // a BFS has at most n layers: the counters are inconsistent
        r.status = BFS_ERR_CUDA;
        go = false;
    }
    if (!go) {
        const bool fill = r.status == BFS_OK && !r.filled;
        r.done = 1;
        if (fill) {
            r.filled = 1;
            r.kernels += 1;
        }
        cudaGraphSetConditional(s.h_case, GL_CASES);
        cudaGraphSetConditional(s.h_fill, fill ? 1u : 0u);
        cudaGraphSetConditional(s.h_loop, 0u);
        return;
    }
    if (r.iter >= kGlCap) {  // this launch is done; the host launches the graph again
        cudaGraphSetConditional(s.h_case, GL_CASES);
        cudaGraphSetConditional(s.h_loop, 0u);
        return;
    }
    const int d = r.d;
    const int cur_bu = decide(s.cfg, r.cur_bu, d, s.n, r.n_f, r.m_f, r.n_u, r.m_u);
    r.cur_bu = cur_bu;
    r.degsum += r.m_f;
    r.sc = s.trace + (d % kRing) * kFields;
    r.sn = s.trace + ((d + 1) % kRing) * kFields;
    r.sz = s.trace + ((d + 2) % kRing) * kFields;
    r.front = (d & 1) ? s.bm_b : s.bm_a;
    r.next = (d & 1) ? s.bm_a : s.bm_b;
    r.q_cur = (d & 1) ? s.q_b : s.q_a;
    r.q_next = (d & 1) ? s.q_a : s.q_b;
    unsigned c;
    int nk;
    r.converted = 0;
    if (!cur_bu) {
        r.queue_mode = r.m_f <= kQueueModeMaxEdges ? 1 : 0;
        r.defer = td_defer(r.queue_mode, r.n_u - s.deg0, s.nw);
        const int64_t pw = (r.n_f + s.td_warps - 1) / s.td_warps;
        r.per_warp = (int)(pw < 1 ? 1 : (pw > 32 ? 32 : pw));
        int64_t gd = r.m_f / s.td_warps;
        if (gd < 4 * (int64_t)s.cfg.td_warp_degree) gd = 4 * (int64_t)s.cfg.td_warp_degree;
        if (gd > s.cfg.td_grid_degree) gd = s.cfg.td_grid_degree;
        r.grid_deg = gd;
        const int b2q = r.have_queue ? 0 : 1, big = r.m_f >= gd ? 1 : 0;
        r.converted = b2q;
        c = GL_TD + b2q + 2 * big + 4 * r.defer;
        nk = 2 + b2q + big + r.defer;
    } else {
        const int64_t active = r.n_u - s.deg0;
        const int fill = r.filled ? 0 : 1;
        if (s.cfg.bu_list_percent > 0 && active * 100 <= (int64_t)s.cfg.bu_list_percent * s.n) {
            r.converted = 2;
            c = fill ? GL_LIST_FILL : GL_LIST;
            nk = 3 + fill;
        } else if (s.two_pass) {
            r.converted = 3;
            r.init_out = fill;
            c = GL_TWO;
            nk = 3;
        } else {
            c = fill ? GL_ONE_FILL : GL_ONE;
            nk = 1 + fill;
        }
        r.filled = 1;
    }
    r.pending = 1;
    r.iter += 1;
    r.kernels += nk;
    cudaGraphSetConditional(s.h_case, c);
    cudaGraphSetConditional(s.h_loop, 1u);
}

// Layer kernels of the graph loop: the host loop's phases with the arguments
// of the planned layer.
__global__ void __launch_bounds__(kBlock) gl_b2q_kernel(GlStatic s) {
    const GlRun &r = *s.run;
    b2q_phase<false>(r.front, s.nw, r.q_cur, (unsigned long long *)(r.sc + T_CONV));
}

__global__ void __launch_bounds__(kBlock) gl_clear_kernel(GlStatic s) {
    uint32_t *next = s.run->next;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.nw_pad; i += stride)
        next[i] = 0u;
}

__device__ __forceinline__ TdArgs gl_td_args(const GlStatic &s, const GlRun &r) {
    return TdArgs{s.off, s.idx, s.visited, r.next, r.parent, r.level, r.q_next,
                  (unsigned long long *)(r.sn + T_NF), r.d + 1, r.queue_mode, s.cfg.td_claim,
                  r.defer};
}

__global__ void __launch_bounds__(kBlock, 4) gl_td_kernel(GlStatic s) {
    const GlRun &r = *s.run;
    td_phase<false>(gl_td_args(s, r), r.q_cur, r.n_f, r.per_warp, s.big,
                    (unsigned long long *)(r.sc + T_BIG), (unsigned long long *)(r.sn + T_MF),
                    s.cfg.td_warp_degree, r.grid_deg, r.sz);
}

__global__ void __launch_bounds__(kBlock, 5) gl_td_big_kernel(GlStatic s) {
    const GlRun &r = *s.run;
    td_big_phase<false>(gl_td_args(s, r), s.big, (const unsigned long long *)(r.sc + T_BIG),
                        (unsigned long long *)(r.sn + T_MF));
}

__global__ void __launch_bounds__(kBlock) gl_td_post_kernel(GlStatic s) {
    const GlRun &r = *s.run;
    td_post_phase<false>(s.off, r.next, s.nw, r.level, r.d + 1,
                         (unsigned long long *)(r.sn + T_NF), (unsigned long long *)(r.sn + T_MF));
}

__global__ void gl_fill_kernel(GlStatic s) {
    const GlRun &r = *s.run;
    out_fill_phase(s.n, r.root, s.visited, s.base_vis, r.level, r.parent);
}

template <bool PEND>
__global__ void __launch_bounds__(kBlock) gl_bits_list_kernel(GlStatic s) {
    const GlRun &r = *s.run;
    bits_list_phase<false>(PEND ? s.pend : s.visited, PEND ? 0u : ~0u, s.nw, r.q_next,
                           (unsigned long long *)(r.sc + T_ULIST));
}

template <bool HEADED>
__global__ void __launch_bounds__(kBlock, 5) gl_bu_list_kernel(GlStatic s) {
    const GlRun &r = *s.run;
    bu_list_phase<false>(s.off, s.idx, HEADED ? s.head : nullptr, HEADED ? s.hskip : 0, r.q_next,
                         (const unsigned long long *)(r.sc + T_ULIST), s.visited, r.front, r.next,
                         r.parent, r.level, r.d + 1, s.cfg.bu_probe, (unsigned long long *)r.sn,
                         r.sz);
}

__global__ void __launch_bounds__(kBlock, 4) gl_bu_hub_kernel(GlStatic s) {
    const GlRun &r = *s.run;
    bu_hub_phase<false>(s.head, s.nw_pad, s.visited, r.front, r.next, s.pend, r.parent, r.level,
                        r.d + 1, (unsigned long long *)r.sn, r.sz, r.init_out, s.base_vis, s.n,
                        r.root);
}

template <int W, int CH, bool HEAD>
__global__ void __launch_bounds__(kBlock, 4) gl_bu_kernel(GlStatic s) {
    const GlRun &r = *s.run;
    bu_phase<W, CH, HEAD, false>(s.off, s.idx, s.head, s.nw_pad, s.visited, r.front, r.next,
                                 r.parent, r.level, r.d + 1, s.cfg.bu_probe,
                                 (unsigned long long *)r.sn, r.sz, s.bu_span_w, s.hskip);
}

void destroy_graph_loop(bfs_graph *g) {
    if (g->gl_exec) cudaGraphExecDestroy(g->gl_exec);
    if (g->gl_graph) cudaGraphDestroy(g->gl_graph);
    g->gl_exec = nullptr;
    g->gl_graph = nullptr;
}

void free_graph_loop(bfs_graph *g) {
    destroy_graph_loop(g);
    cudaFree(g->gl_mem);
    if (g->h_gl) cudaFreeHost(g->h_gl);
    delete (GlStatic *)g->gl_static;
    g->gl_mem = g->h_gl = g->gl_static = nullptr;
}

// Builds and instantiates the graph for the graph's current configuration.
bfs_status build_graph_loop(bfs_graph *g) {
    const bfs_config &cfg = g->cfg;
    if (!g->gl_mem) {
        GB_CK(dev_malloc(&g->gl_mem, kGlRunBytes + (size_t)kSsMaxRecords * kGlRec * 8));
        GB_CK(host_malloc(&g->h_gl, kGlRunBytes + (size_t)kSsMaxRecords * kGlRec * 8));
    }
    const int bw = cfg.bu_words;
    const int bsel = (bw == 4 ? 2 : bw - 1) + (cfg.bu_head ? 3 : 0);
    const void *one_fn[6] = {(const void *)gl_bu_kernel<1, 4, false>,
                             (const void *)gl_bu_kernel<2, 4, false>,
                             (const void *)gl_bu_kernel<4, 2, false>,
                             (const void *)gl_bu_kernel<1, 4, true>,
                             (const void *)gl_bu_kernel<2, 4, true>,
                             (const void *)gl_bu_kernel<4, 2, true>};
    // resident blocks per SM of the graph's own kernels (their register
    // counts differ from the host loop's kernels)
    auto occ = [](const void *fn, int *out) -> cudaError_t {
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, fn, kBlock, 0);
        if (*out < 1) *out = 1;
        return e;
    };
    int o_td = 1, o_big = 1, o_list = 1, o_hub = 1, o_one = 1;
    GB_CK(occ((const void *)gl_td_kernel, &o_td));
    GB_CK(occ((const void *)gl_td_big_kernel, &o_big));
    GB_CK(occ((const void *)gl_bu_list_kernel<true>, &o_list));
    GB_CK(occ((const void *)gl_bu_hub_kernel, &o_hub));
    GB_CK(occ(one_fn[bsel], &o_one));
    const int64_t bu_full = (int64_t)sm_count() * o_one;
    const int64_t td_full = (int64_t)sm_count() * o_td;
    if (!g->gl_static) g->gl_static = new GlStatic;
    GlStatic &s = *(GlStatic *)g->gl_static;
    memset(&s, 0, sizeof s);
    s.off = g->off;
    s.idx = g->idx;
    s.head = cfg.bu_head ? g->head : nullptr;
    s.hskip = cfg.bu_head == 1 ? 1 : 0;
    s.base_vis = g->base_vis;
    s.visited = g->visited;
    s.bm_a = g->bm_a;
    s.bm_b = g->bm_b;
    s.pend = g->pend;
    s.q_a = g->q_a;
    s.q_b = g->q_b;
    s.big = g->big;
    s.trace = g->trace;
    s.run = (GlRun *)g->gl_mem;
    s.rec = (int64_t *)((char *)g->gl_mem + kGlRunBytes);
    s.n = g->n;
    s.nnz = g->nnz;
    s.nw = g->nw;
    s.nw_pad = g->nw_pad;
    s.deg0 = g->deg0;
    s.td_warps = td_full * (kBlock / 32);
    s.two_pass = cfg.bu_head == 2 &&
                 g->nw >= (int64_t)8 * sm_count() * g->bu_hub_blocks_per_sm * (kBlock / 32);
    s.bu_span_w = bu_span(g->nw_pad >> 5, bw, bu_full * (kBlock / 32));
    s.cfg = cfg;

    cudaGraph_t gr = nullptr;
    GB_CK(cudaGraphCreate(&gr, 0));
    struct Guard {
        cudaGraph_t &gr;
        ~Guard() {
            if (gr) cudaGraphDestroy(gr);
        }
    } guard{gr};
    GB_CK(cudaGraphConditionalHandleCreate(&s.h_loop, gr, 1, cudaGraphCondAssignDefault));
    GB_CK(cudaGraphConditionalHandleCreate(&s.h_fill, gr, 0, cudaGraphCondAssignDefault));
    void *args[] = {&s};
    auto kernel = [&](cudaGraph_t in, cudaGraphNode_t *dep, const void *fn, int grid,
                      int block) -> cudaError_t {
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof kp);
        kp.func = const_cast<void *>(fn);
        kp.gridDim = dim3(grid);
        kp.blockDim = dim3(block);
        kp.kernelParams = args;
        cudaGraphNode_t node;
        const cudaError_t e = cudaGraphAddKernelNode(&node, in, *dep ? dep : nullptr, *dep ? 1 : 0,
                                                     &kp);
        *dep = node;
        return e;
    };
    auto conditional = [&](cudaGraph_t in, cudaGraphNode_t *dep, cudaGraphConditionalHandle h,
                           cudaGraphConditionalNodeType type, unsigned size,
                           cudaGraph_t **bodies) -> cudaError_t {
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = type;
        np.conditional.size = size;
        cudaGraphNode_t node;
        const cudaError_t e = cudaGraphAddNode(&node, in, *dep ? dep : nullptr, nullptr,
                                               *dep ? 1 : 0, &np);
        *dep = node;
        *bodies = np.conditional.phGraph_out;
        return e;
    };
    cudaGraphNode_t top = nullptr;
    GB_CK(kernel(gr, &top, (const void *)gl_begin_kernel, 1, 32));
    cudaGraph_t *loop_body = nullptr;
    GB_CK(conditional(gr, &top, s.h_loop, cudaGraphCondTypeWhile, 1, &loop_body));
    cudaGraph_t body = loop_body[0];
    GB_CK(cudaGraphConditionalHandleCreate(&s.h_case, body, GL_CASES, cudaGraphCondAssignDefault));
    cudaGraphNode_t step = nullptr;
    GB_CK(kernel(body, &step, (const void *)gl_step_kernel, 1, 32));
    cudaGraph_t *cases = nullptr;
    GB_CK(conditional(body, &step, s.h_case, cudaGraphCondTypeSwitch, GL_CASES, &cases));

    const int g_b2q = grid_cap(g->nw, kBlock * 4, 8);
    const int g_clear = grid_cap(g->nw_pad, kBlock, 8);
    const int g_td = (int)std::max<int64_t>(1, td_full);
    const int g_big = (int)std::max<int64_t>(1, (int64_t)sm_count() * o_big);
    const int g_post = grid_cap(g->nw, kBlock / 4, 8);
    const int g_fill = grid_cap(g->n, kBlock, 8);
    const int g_bits = grid_cap(g->nw, kBlock * 4, 8);
    const int g_list = (int)std::max<int64_t>(1, (int64_t)sm_count() * o_list);
    const int g_hub = grid_cap(g->nw_pad, kBlock / 32 * 8, o_hub);
    const int g_one = (int)std::max<int64_t>(
        1, std::min<int64_t>((g->nw_pad >> 5) * (32 / s.bu_span_w) / (kBlock / 32) + 1, bu_full));
    for (unsigned c = 0; c < GL_CASES; ++c) {
        cudaGraph_t b = cases[c];
        cudaGraphNode_t t = nullptr;
        if (c < GL_LIST) {
            if (c & 1) GB_CK(kernel(b, &t, (const void *)gl_b2q_kernel, g_b2q, kBlock));
            GB_CK(kernel(b, &t, (const void *)gl_clear_kernel, g_clear, kBlock));
            GB_CK(kernel(b, &t, (const void *)gl_td_kernel, g_td, kBlock));
            if (c & 2) GB_CK(kernel(b, &t, (const void *)gl_td_big_kernel, g_big, kBlock));
            if (c & 4) GB_CK(kernel(b, &t, (const void *)gl_td_post_kernel, g_post, kBlock));
        } else if (c == GL_LIST || c == GL_LIST_FILL) {
            if (c == GL_LIST_FILL) GB_CK(kernel(b, &t, (const void *)gl_fill_kernel, g_fill, kBlock));
            GB_CK(kernel(b, &t, (const void *)gl_clear_kernel, g_clear, kBlock));
            GB_CK(kernel(b, &t, (const void *)gl_bits_list_kernel<false>, g_bits, kBlock));
            GB_CK(kernel(b, &t, (const void *)gl_bu_list_kernel<true>, g_list, kBlock));
        } else if (c == GL_TWO) {
            GB_CK(kernel(b, &t, (const void *)gl_bu_hub_kernel, g_hub, kBlock));
            GB_CK(kernel(b, &t, (const void *)gl_bits_list_kernel<true>, g_bits, kBlock));
            GB_CK(kernel(b, &t, (const void *)gl_bu_list_kernel<false>, g_list, kBlock));
        } else {
            if (c == GL_ONE_FILL) GB_CK(kernel(b, &t, (const void *)gl_fill_kernel, g_fill, kBlock));
            GB_CK(kernel(b, &t, one_fn[bsel], g_one, kBlock));
        }
    }
    cudaGraph_t *fill_body = nullptr;
    GB_CK(conditional(gr, &top, s.h_fill, cudaGraphCondTypeIf, 1, &fill_body));
    cudaGraphNode_t f = nullptr;
    GB_CK(kernel(fill_body[0], &f, (const void *)gl_fill_kernel, g_fill, kBlock));
    GB_CK(cudaGraphInstantiate(&g->gl_exec, gr, 0));
    g->gl_graph = gr;
    gr = nullptr;  // owned by g now
    return BFS_OK;
}

// Runs the traversal through the graph loop (init_kernel has already run on
// `st`) and reads back the per-layer records.
bfs_status run_graph_loop(bfs_graph *g, int32_t *level, int32_t *parent, int32_t root,
                          int filled, cudaStream_t st) {
    if (g->gl_exec && memcmp(&((const GlStatic *)g->gl_static)->cfg, &g->cfg, sizeof g->cfg) != 0)
        destroy_graph_loop(g);  // built for another configuration
    if (!g->gl_exec) {
        const bfs_status bs = build_graph_loop(g);
        if (bs != BFS_OK) return bs;
    }
    const GlStatic &s = *(const GlStatic *)g->gl_static;
    GB_LAUNCH(gl_start_kernel, 1, 32, 0, st, s, level, parent, root, filled);
    constexpr int64_t kFirst = 64;  // records fetched with the state
    const size_t first_bytes = kGlRunBytes + (size_t)kFirst * kGlRec * 8;
    const GlRun *hr = (const GlRun *)g->h_gl;
    int64_t counted = 0;
    for (int64_t launch = 0;; ++launch) {
        if (launch > g->n / kGlCap + 2) {
            set_error("bfs_run: internal error, graph loop did not finish after %lld launches",
                      (long long)launch);
            cudaStreamSynchronize(st);
            return BFS_ERR_INTERNAL;
        }
        GB_CK(cudaGraphLaunch(g->gl_exec, st));
        GB_CK(cudaMemcpyAsync(g->h_gl, g->gl_mem, first_bytes, cudaMemcpyDeviceToHost, st));
        GB_CK(cudaStreamSynchronize(st));
        count_launch((int)(hr->kernels - counted) + 1);  // layer kernels and gl_begin_kernel
        counted = hr->kernels;
        if (hr->done || hr->status != BFS_OK) break;
    }
    if (hr->status != BFS_OK) {
        set_error("bfs_run: the graph loop stopped (status %d)", hr->status);
        return (bfs_status)hr->status;
    }
    const int64_t L = hr->d;
    if (L > kFirst) {
        const int64_t more = std::min<int64_t>(L, kSsMaxRecords) - kFirst;
        GB_CK(cudaMemcpyAsync((char *)g->h_gl + first_bytes, (char *)g->gl_mem + first_bytes,
                              (size_t)more * kGlRec * 8, cudaMemcpyDeviceToHost, st));
        GB_CK(cudaStreamSynchronize(st));
    }
    const int64_t *recs = (const int64_t *)((const char *)g->h_gl + kGlRunBytes);
    for (int64_t d = 0; d < L && d < kSsMaxRecords; ++d) {
        const int64_t *rec = recs + d * kGlRec;
        bfs_layer_stats ls;
        memset(&ls, 0, sizeof ls);
        ls.direction = (int32_t)rec[0];
        ls.converted = (int32_t)rec[1];
        ls.n_f = rec[2];
        ls.m_f = rec[3];
        ls.n_u = rec[4];
        ls.m_u = rec[5];
        ls.examined = rec[6];
        ls.found = rec[7];
        ls.hub_found = rec[8];
        g->last.push_back(ls);
    }
    g->last_component_edges = hr->degsum / 2;
    return BFS_OK;
}

bool is_host_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

void free_graph(bfs_graph *g) {
    if (!g) return;
    free_ms_state(g);
    cudaFree(g->off_own);
    cudaFree(g->idx_own);
    cudaFree(g->visited);
    cudaFree(g->base_vis);
    cudaFree(g->head);
    cudaFree(g->hubc);
    cudaFree(g->wrank);
    cudaFree(g->wmeta);
    cudaFree(g->comp_in);
    cudaFree(g->pctl);
    if (g->h_pctl) cudaFreeHost(g->h_pctl);
    free_graph_loop(g);
    cudaFree(g->bm_a);
    cudaFree(g->bm_b);
    cudaFree(g->ring);
    cudaFree(g->pend);
    cudaFree(g->q_a);
    cudaFree(g->q_b);
    cudaFree(g->big);
    cudaFree(g->parent_scratch);
    cudaFree(g->level_scratch);
    if (g->copy_st) cudaStreamSynchronize(g->copy_st);
    for (int i = 0; i < 2; ++i) {
        cudaFree(g->hout_level[i]);
        cudaFree(g->hout_parent[i]);
        if (g->hout_done[i]) cudaEventDestroy(g->hout_done[i]);
    }
    if (g->hout_ready) cudaEventDestroy(g->hout_ready);
    if (g->copy_st) cudaStreamDestroy(g->copy_st);
    cudaFree(g->trace);
    cudaFree(g->misc);
    if (g->h_slot) cudaFreeHost(g->h_slot);
    if (g->h_pub) cudaFreeHost(g->h_pub);
    for (cudaEvent_t e : g->events) cudaEventDestroy(e);
    delete g;
}

// Head records for the bottom-up probe (kind 1: the row's first entry, kind
// 2: the hub), built with the graph when its configuration asks for them,
// else on first use, and rebuilt when the kind changes.
bfs_status build_head(bfs_graph *g, int kind, cudaStream_t st) {
    // nw_pad * 32 records: the streaming sweep copies whole tiles of 1024;
    // the records past n hold {-1, -1} (no probe)
    const size_t recs = (size_t)g->nw_pad * 32;
    if (!g->head) {
        GB_CK(dev_malloc(&g->head, recs * sizeof(int2)));
        GB_CK(cudaMemsetAsync(g->head + g->n, 0xff, (recs - (size_t)g->n) * sizeof(int2), st));
    }
    if (kind == 1)
        GB_LAUNCH(head_kernel, grid_cap(g->n, kBlock, 8), kBlock, 0, st, g->off, g->idx, g->n,
                  g->head);
    else
        GB_LAUNCH(hub_head_kernel, grid_cap(g->n, kBlock / 32, 8), kBlock, 0, st, g->off,
                  g->idx, g->n, g->head);
    if (kind == 2 && !g->hubc) {
        // the compact 4-byte hub records the host loop's two-pass sweeps read
        g->n1 = g->n - g->deg0;
        GB_CK(dev_malloc(&g->wrank, (size_t)(g->nw_pad + 1) * 4));
        GB_CK(dev_malloc(&g->hubc, (size_t)(g->n1 + 16) * 4));
        GB_CK(cudaMemsetAsync(g->hubc + g->n1, 0xff, 16 * 4, st));
        GB_LAUNCH(word_rank_kernel, 1, 1024, 0, st, g->base_vis, g->nw_pad, g->wrank);
        GB_LAUNCH(hubc_kernel, grid_cap(g->nw_pad, kBlock / 32, 8), kBlock, 0, st, g->head,
                  g->base_vis, g->wrank, g->nw_pad, g->hubc);
        GB_CK(dev_malloc(&g->wmeta, (size_t)g->nw_pad * sizeof(uint2)));
        GB_LAUNCH(wmeta_kernel, grid_cap(g->nw_pad, kBlock, 8), kBlock, 0, st, g->base_vis,
                  g->wrank, g->nw_pad, g->wmeta);
    }
    g->head_kind = kind;
    return BFS_OK;
}

// Publishes `slot` to the host block and waits for it there: a spin on the
// sequence number in mapped memory instead of a copy plus a stream
// synchronisation (a layer's host round trip is what small layers cost).
// The spin gives up after 5 s and then synchronises the stream, which
// returns the error of a failed kernel; the counters land in g->h_slot.
bfs_status publish_and_wait(bfs_graph *g, const int64_t *slot, cudaStream_t st) {
    const int64_t seq = ++g->pub_seq;
    publish_kernel<<<1, 32, 0, st>>>(slot, g->d_pub, seq);
    count_launch();
    GB_CK(cudaGetLastError());
    volatile int64_t *vp = g->h_pub;
    const auto t0 = std::chrono::steady_clock::now();
    for (long spins = 0; vp[kFields] != seq; ++spins) {
        if ((spins & 1023) == 1023) {
            if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(5)) {
                GB_CK(cudaStreamSynchronize(st));
                if (vp[kFields] != seq) {
                    set_error("bfs_run: the layer counters never arrived");
                    return BFS_ERR_CUDA;
                }
                break;
            }
            if (spins > (1 << 16)) std::this_thread::yield();
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    for (int i = 0; i < kFields; ++i) g->h_slot[i] = vp[i];
    return BFS_OK;
}

}  // namespace
}  // namespace gbfs

using namespace gbfs;

extern "C" BFS_API void bfs_config_default(bfs_config *c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->policy = BFS_POLICY_EDGE;
    c->forced_len = 1;
    // measured best at R-MAT scale 26 with the two-pass bottom-up step
    // (alpha 14 / beta 24: 913 GTEPS; 20 / 200: 939), neutral at scale 20-22
    c->alpha = 20.0;
    c->beta = 200.0;
    c->bu_probe = 8;
    c->td_warp_degree = 32;
    c->td_grid_degree = 1024;
    c->timing = 0;
    c->bu_words = 2;
    c->bu_head = 2;
    c->td_claim = 1;
    c->prune_components = 0;
    c->bu_list_percent = 10;
    c->device_loop = 2;
    // measured at scale 26: 2 stages per warp, every two-pass sweep streamed
    c->hub_stream_stages = 2;
    c->hub_stream_percent = 0;
    // measured at scale 26: 1033 GTEPS storing levels as found, 1007 with the
    // level pass (the first hub sweep writes whole rows anyway, and the pass
    // rewrites every level)
    c->level_pass = 0;
}

extern "C" BFS_API bfs_status bfs_graph_create(const int64_t *offsets, const int32_t *indices,
                                               int64_t n, int64_t nnz, uint32_t flags,
                                               const bfs_config *cfg, bfs_graph **out) {
    clear_error();
    if (!out || !offsets || (nnz > 0 && !indices) || n < 1 || n >= (1ll << 31) || nnz < 0 ||
        ((flags & BFS_BORROW) && !(flags & BFS_DEVICE_PTRS))) {
        set_error("bfs_graph_create: need offsets/indices/out, 1 <= n < 2^31, nnz >= 0; "
                  "BFS_BORROW needs BFS_DEVICE_PTRS");
        return BFS_ERR_INVALID;
    }
    *out = nullptr;
    bfs_config c;
    if (cfg) c = *cfg;
    else bfs_config_default(&c);
    if (!config_ok(c)) {
        set_error("bfs_graph_create: invalid bfs_config");
        return BFS_ERR_INVALID;
    }
    bfs_graph *g = new bfs_graph();
    g->cfg = c;
    g->n = n;
    g->nnz = nnz;
    g->nw = (n + 31) / 32;
    g->nw_pad = ((g->nw + 31) / 32) * 32;
#define GB_CKG(call)                                                    \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) {                                        \
            bfs_status _s = cuda_status(_e, #call, __FILE__, __LINE__); \
            free_graph(g);                                              \
            return _s;                                                  \
        }                                                               \
    } while (0)
    GB_CKG(cudaGetDevice(&g->device));
    if ((flags & BFS_DEVICE_PTRS) && (flags & BFS_BORROW)) {
        g->off = offsets;
        g->idx = indices;
    } else {
        const cudaMemcpyKind kind =
            (flags & BFS_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        GB_CKG(dev_malloc(&g->off_own, (size_t)(n + 1) * 8));
        GB_CKG(dev_malloc(&g->idx_own, (size_t)std::max<int64_t>(nnz, 1) * 4));
        GB_CKG(cudaMemcpy(g->off_own, offsets, (size_t)(n + 1) * 8, kind));
        if (nnz) GB_CKG(cudaMemcpy(g->idx_own, indices, (size_t)nnz * 4, kind));
        g->off = g->off_own;
        g->idx = g->idx_own;
    }
    const size_t bmb = (size_t)g->nw_pad * 4;
    GB_CKG(dev_malloc(&g->visited, bmb));
    GB_CKG(dev_malloc(&g->base_vis, bmb));
    GB_CKG(dev_malloc(&g->bm_a, bmb));
    GB_CKG(dev_malloc(&g->bm_b, bmb));
    GB_CKG(dev_malloc(&g->q_a, (size_t)n * 4));
    GB_CKG(dev_malloc(&g->q_b, (size_t)n * 4));
    GB_CKG(dev_malloc(&g->big, (size_t)n * 4));
    GB_CKG(dev_malloc(&g->trace, (size_t)kRing * kFields * 8));
    GB_CKG(dev_malloc(&g->misc, 64));
    GB_CKG(dev_malloc(&g->pend, bmb));  // two-pass bottom-up: vertices whose hub missed
    GB_CKG(host_malloc(&g->h_slot, kFields * 8));
    GB_CKG(host_malloc((void **)&g->h_pub, (kFields + 1) * 8, cudaHostAllocMapped));
    GB_CKG(cudaHostGetDevicePointer((void **)&g->d_pub, g->h_pub, 0));
    g->h_pub[kFields] = 0;
    if (flags & (BFS_VALIDATE | BFS_VALIDATE_SYMMETRIC)) {
        int *bad = nullptr, hbad = 0;
        GB_CKG(dev_malloc(&bad, sizeof(int)));
        cudaMemset(bad, 0, sizeof(int));
        validate_kernel<<<grid_cap(std::max(n, nnz), kBlock, 8), kBlock>>>(g->off, g->idx, n, nnz,
                                                                           bad);
        count_launch();
        cudaError_t e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && !hbad && (flags & BFS_VALIDATE_SYMMETRIC)) {
            // the row bounds and indices it follows were checked above
            symmetric_kernel<<<grid_cap(n * 32, kBlock, 8), kBlock>>>(g->off, g->idx, n, bad);
            count_launch();
            e = cudaMemcpy(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && hbad) hbad = 2;
        }
        cudaFree(bad);
        GB_CKG(e);
        if (hbad) {
            free_graph(g);
            set_error(hbad == 2 ? "bfs_graph_create: CSR failed validation (a row not strictly "
                                  "ascending, or an entry without its reverse entry)"
                                : "bfs_graph_create: CSR failed validation (offsets or indices "
                                  "out of range)");
            return BFS_ERR_INVALID;
        }
    }
    base_vis_kernel<<<grid_cap(g->nw_pad, kBlock, 8), kBlock>>>(g->off, n, g->nw_pad, g->base_vis);
    count_launch();
    {  // degree-0 vertices = set bits of base_vis minus the padding bits
        unsigned long long *cnt = nullptr, hc = 0;
        GB_CKG(dev_malloc(&cnt, 8));
        cudaMemset(cnt, 0, 8);
        count_bits_kernel<<<grid_cap(g->nw_pad, kBlock, 8), kBlock>>>(g->base_vis, g->nw_pad, cnt);
        count_launch();
        cudaError_t e = cudaMemcpy(&hc, cnt, 8, cudaMemcpyDeviceToHost);
        cudaFree(cnt);
        GB_CKG(e);
        g->deg0 = (int64_t)hc - (g->nw_pad * 32 - n);
    }
    GB_CKG(cudaGetLastError());
    GB_CKG(cudaDeviceSynchronize());
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->bu_blocks_per_sm[0], BU1, kBlock, 0));
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->bu_blocks_per_sm[1], BU2, kBlock, 0));
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->bu_blocks_per_sm[2], BU4, kBlock, 0));
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->bu_blocks_per_sm[3], BU1H, kBlock, 0));
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->bu_blocks_per_sm[4], BU2H, kBlock, 0));
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->bu_blocks_per_sm[5], BU4H, kBlock, 0));
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->td_blocks_per_sm, td_kernel, kBlock, 0));
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->bu_list_blocks_per_sm, bu_list_kernel,
                                                         kBlock, 0));
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->bu_hub_blocks_per_sm, bu_hub_kernel,
                                                         kBlock, 0));
    GB_CKG(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g->hubc_blocks_per_sm, bu_hubc_kernel,
                                                         kBlock, 0));
    if (g->cfg.bu_head) {
        const bfs_status hs = build_head(g, g->cfg.bu_head, 0);
        if (hs != BFS_OK) {
            free_graph(g);
            return hs;
        }
        GB_CKG(cudaDeviceSynchronize());
    }
#undef GB_CKG
    *out = g;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_graph_set_config(bfs_graph *g, const bfs_config *cfg) {
    clear_error();
    if (!g) {
        set_error("bfs_graph_set_config: null graph");
        return BFS_ERR_INVALID;
    }
    bfs_config c;
    if (cfg) c = *cfg;
    else bfs_config_default(&c);
    if (!config_ok(c)) {
        set_error("bfs_graph_set_config: invalid bfs_config");
        return BFS_ERR_INVALID;
    }
    g->cfg = c;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_graph_info(const bfs_graph *g, const int64_t **offsets,
                                             const int32_t **indices, int64_t *n, int64_t *nnz) {
    clear_error();
    if (!g) {
        set_error("bfs_graph_info: null graph");
        return BFS_ERR_INVALID;
    }
    if (offsets) *offsets = g->off;
    if (indices) *indices = g->idx;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_graph_destroy(bfs_graph *g) {
    clear_error();
    free_graph(g);
    return BFS_OK;
}

// Everything bfs_run would otherwise allocate or build on first use under
// the graph's current configuration, for outputs in host memory (host_out)
// or not, and with or without a caller-given parent array: output scratch or
// the host_async output pairs and copy stream, the head records of the
// configured kind, the component mask (prune_components, one traversal), the
// device-loop records, the graph loop's graph, the rows-sorted check of
// parent_min and the streaming sweep's shared-memory limit.
static bfs_status prepare(bfs_graph *g, bool host_out, bool have_parent, void *stream) {
    cudaStream_t st = as_stream(stream);
    const bfs_config &cfg = g->cfg;
    const int64_t n = g->n;
    if (host_out && cfg.host_async) {
        if (!g->copy_st) {
            GB_CK(cudaStreamCreateWithFlags(&g->copy_st, cudaStreamNonBlocking));
            GB_CK(cudaEventCreateWithFlags(&g->hout_ready, cudaEventDisableTiming));
            for (int i = 0; i < 2; ++i)
                GB_CK(cudaEventCreateWithFlags(&g->hout_done[i], cudaEventDisableTiming));
        }
        for (int i = 0; i < 2; ++i)
            if (!g->hout_level[i]) {
                GB_CK(dev_malloc(&g->hout_level[i], (size_t)n * 4));
                GB_CK(dev_malloc(&g->hout_parent[i], (size_t)n * 4));
            }
    } else if (host_out) {
        if (!g->level_scratch) GB_CK(dev_malloc(&g->level_scratch, (size_t)n * 4));
        have_parent = false;  // the parent is computed in scratch and copied
    }
    if (!have_parent && !(host_out && cfg.host_async) && !g->parent_scratch)
        GB_CK(dev_malloc(&g->parent_scratch, (size_t)n * 4));
    if (cfg.prune_components && g->comp_rep < 0) {
        // The component of the highest-degree vertex, found once by one
        // traversal without pruning, kept as a bitmap.
        unsigned long long *best = reinterpret_cast<unsigned long long *>(g->misc);
        unsigned long long hb = 0;
        GB_CK(cudaMemsetAsync(best, 0, 8, st));
        GB_LAUNCH(max_degree_kernel, grid_cap(n, kBlock, 8), kBlock, 0, st, g->off, n, best);
        GB_CK(cudaMemcpyAsync(&hb, best, 8, cudaMemcpyDeviceToHost, st));
        GB_CK(cudaStreamSynchronize(st));
        const int32_t rep = (int32_t)(0xffffffffull - (hb & 0xffffffffull));
        if (!g->comp_in) GB_CK(dev_malloc(&g->comp_in, (size_t)g->nw_pad * 4));
        if (!g->level_scratch) GB_CK(dev_malloc(&g->level_scratch, (size_t)n * 4));
        if (!g->parent_scratch) GB_CK(dev_malloc(&g->parent_scratch, (size_t)n * 4));
        const bfs_config saved = g->cfg;
        g->cfg.prune_components = 0;
        g->cfg.timing = 0;
        const bfs_status s = bfs_run(g, rep, g->level_scratch, g->parent_scratch, stream);
        g->cfg = saved;
        if (s != BFS_OK) return s;
        GB_LAUNCH(reached_bits_kernel, grid_cap(g->nw_pad, kBlock, 8), kBlock, 0, st,
                  g->level_scratch, n, g->nw_pad, g->comp_in);
        GB_CK(cudaStreamSynchronize(st));
        g->comp_rep = rep;
    }
    if (cfg.bu_head && g->head_kind != cfg.bu_head) {
        const bfs_status hs = build_head(g, cfg.bu_head, st);
        if (hs != BFS_OK) return hs;
    }
    const bool dev_loop = cfg.device_loop == 1 || cfg.device_loop == 4 ||
                          (cfg.device_loop == 2 && n <= kDeviceLoopAutoMaxN);
    if (dev_loop && !g->pctl) {
        GB_CK(dev_malloc(&g->pctl, kPctlSsBytes));
        GB_CK(host_malloc(&g->h_pctl, kPctlSsBytes));
    }
    const bool host_loop = !(cfg.device_loop == 1 || cfg.device_loop == 4 ||
                             (cfg.device_loop == 2 && n <= kDeviceLoopAutoMaxN) ||
                             (cfg.device_loop == 3 && cfg.timing == 0));
    if (cfg.level_pass && host_loop && !g->ring)
        GB_CK(dev_malloc(&g->ring, (size_t)kLevelRing * g->nw_pad * 4));
    if (cfg.device_loop == 3 && cfg.timing == 0) {
        if (g->gl_exec &&
            memcmp(&((const GlStatic *)g->gl_static)->cfg, &g->cfg, sizeof g->cfg) != 0)
            destroy_graph_loop(g);  // built for another configuration
        if (!g->gl_exec) {
            const bfs_status bs = build_graph_loop(g);
            if (bs != BFS_OK) return bs;
        }
    }
    if (cfg.parent_min && g->rows_sorted < 0) {  // checked once per graph
        int *flag = reinterpret_cast<int *>(g->misc);
        int h = 1;
        GB_CK(cudaMemcpyAsync(flag, &h, 4, cudaMemcpyHostToDevice, st));
        GB_LAUNCH(rows_sorted_kernel, grid_cap(n, kBlock, 8), kBlock, 0, st, g->off, g->idx, n,
                  flag);
        GB_CK(cudaMemcpyAsync(&h, flag, 4, cudaMemcpyDeviceToHost, st));
        GB_CK(cudaStreamSynchronize(st));
        g->rows_sorted = h;
    }
    if (cfg.hub_stream_stages > 0 && g->hub_stream_occ_stages != cfg.hub_stream_stages) {
        const size_t smem = hub_stream_smem_bytes(cfg.hub_stream_stages);
        for (int init = 0; init < 2; ++init)
            GB_CK(cudaFuncSetAttribute(hub_stream_fn(cfg.hub_stream_stages, init != 0),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &g->hub_stream_occ, hub_stream_fn(cfg.hub_stream_stages, true), kBlock, smem));
        g->hub_stream_occ_stages = cfg.hub_stream_stages;
    }
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_graph_reserve(bfs_graph *g, uint32_t flags, void *stream) {
    clear_error();
    if (!g || (flags & ~(BFS_RESERVE_HOST_OUT | BFS_RESERVE_NO_PARENT))) {
        set_error("bfs_graph_reserve: need a graph and known flags");
        return BFS_ERR_INVALID;
    }
    const bfs_status s = prepare(g, (flags & BFS_RESERVE_HOST_OUT) != 0,
                                 (flags & BFS_RESERVE_NO_PARENT) == 0, stream);
    if (s == BFS_OK) GB_CK(cudaStreamSynchronize(as_stream(stream)));
    return s;
}

extern "C" BFS_API bfs_status bfs_run(bfs_graph *g, int32_t root, int32_t *level_out,
                                      int32_t *parent_out, void *stream) {
    clear_error();
    if (!g || !level_out || root < 0 || root >= g->n) {
        set_error("bfs_run: need a graph, level_out and 0 <= root < n");
        return BFS_ERR_INVALID;
    }
    cudaStream_t st = as_stream(stream);
    const int64_t n = g->n;
    const bool host_out = is_host_ptr(level_out);
    if (parent_out && is_host_ptr(parent_out) != host_out) {
        set_error("bfs_run: level_out and parent_out must both be host or both be device memory");
        return BFS_ERR_INVALID;
    }
    {
        const bfs_status ps = prepare(g, host_out, parent_out != nullptr, stream);
        if (ps != BFS_OK) return ps;
    }
    int32_t *level = level_out, *parent = parent_out;
    const bool async_out = host_out && g->cfg.host_async;
    int slot = 0;
    if (async_out) {
        // device outputs used in turn: pair `slot` was last copied two calls ago
        slot = g->hout_turn;
        g->hout_turn ^= 1;
        GB_CK(cudaEventSynchronize(g->hout_done[slot]));
        level = g->hout_level[slot];
        parent = g->hout_parent[slot];
    } else if (host_out) {
        level = g->level_scratch;
        parent = nullptr;
    }
    if (!parent) parent = g->parent_scratch;
    const bfs_config &cfg = g->cfg;
    const bool timing = cfg.timing != 0;
    const bool all_events = cfg.timing == 1;  // 2: only around the hub sweeps
    auto event = [&](size_t i) -> cudaEvent_t {
        while (g->events.size() <= i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            g->events.push_back(e);
        }
        return g->events[i];
    };

    const int hskip = cfg.bu_head == 1 ? 1 : 0;
    g->last.clear();
    int32_t *q_cur = g->q_a, *q_next = g->q_b;
    const bool dev_loop = cfg.device_loop == 1 || (cfg.device_loop == 2 && n <= kDeviceLoopAutoMaxN);
    // the graph loop has no per-layer events: timed runs take the host loop
    const bool graph_loop = cfg.device_loop == 3 && !timing;
    // level pass (host loop): the frontiers stay in the ring, levels are
    // written once at the end (or at the flush before the ring wraps)
    const bool lpass = cfg.level_pass && !dev_loop && !graph_loop && cfg.device_loop != 4;
    uint32_t *front = lpass ? g->ring : g->bm_a;
    uint32_t *next = lpass ? g->ring + g->nw_pad : g->bm_b;
    // dense bottom-up layers run in two passes on hub records
    const bool two_pass =
        cfg.bu_head == 2 &&
        g->nw >= (int64_t)8 * sm_count() * g->bu_hub_blocks_per_sm * (kBlock / 32);
    // Without the CAS claim on parent nothing reads the outputs before they
    // are written, so the -1 fill can wait for the first hub sweep (which
    // writes every vertex not reached before it, mostly whole sectors).
    const bool fuse_init = !dev_loop && two_pass && cfg.td_claim == 1 && !cfg.prune_components;
    GB_LAUNCH(init_kernel, grid_cap(std::max(n, g->nw_pad), kBlock, 8), kBlock, 0, st, n,
              g->nw_pad, root, g->off, g->base_vis, cfg.prune_components ? g->comp_in : nullptr,
              level, parent, g->visited, front, q_cur, g->trace, fuse_init ? 0 : 1);
    if (dev_loop) {
        const bfs_status ds = run_device_loop(g, level, parent, st);
        if (ds != BFS_OK) return ds;
    } else if (graph_loop) {
        const bfs_status gs = run_graph_loop(g, level, parent, root, fuse_init ? 0 : 1, st);
        if (gs != BFS_OK) return gs;
    } else {
        // hybrid: stretches of top-down layers run in the persistent kernel
        // (no host round trip per layer), bottom-up layers from the host
        const bool hybrid = cfg.device_loop == 4 && !all_events;
        int64_t n_f = 1, m_f = 0, n_u = n - 1, m_u = 0;
        int cur_bu = 0;
        bool have_queue = true;
        int64_t degree_sum = 0;
        int d_first = 0;
        // takes over the state a device stretch ended in
        auto adopt = [&](const LoopState &s2) {
            d_first = (int)s2.d;
            n_f = s2.n_f;
            m_f = s2.m_f;
            n_u = s2.n_u;
            m_u = s2.m_u;
            degree_sum = s2.degsum;
            cur_bu = s2.cur_bu;
            have_queue = s2.have_queue != 0;
            front = (s2.d & 1) ? g->bm_b : g->bm_a;
            next = (s2.d & 1) ? g->bm_a : g->bm_b;
            q_cur = (s2.d & 1) ? g->q_b : g->q_a;
            q_next = (s2.d & 1) ? g->q_a : g->q_b;
        };
        if (hybrid) {
            LoopState s0;
            s0.n_u = n - 1;  // m_f < 0: the kernel reads the root's degree
            const bfs_status ss = run_device_segment(g, level, parent, st, s0, true);
            if (ss != BFS_OK) return ss;
            adopt(s0);
        } else {
            const bfs_status ps = publish_and_wait(g, g->trace, st);
            if (ps != BFS_OK) return ps;
            m_f = g->h_slot[T_MF];
            m_u = g->nnz - m_f;
        }
        const int bw = cfg.bu_words;
        const int bsel = (bw == 4 ? 2 : bw - 1) + (cfg.bu_head ? 3 : 0);
        const int64_t bu_full = (int64_t)sm_count() * g->bu_blocks_per_sm[bsel];
        const int bu_span_w = bu_span(g->nw_pad >> 5, bw, bu_full * (kBlock / 32));
        const int bu_grid = (int)std::max<int64_t>(
            1, std::min<int64_t>((g->nw_pad >> 5) * (32 / bu_span_w) / (kBlock / 32) + 1,
                                 bu_full));
        const int64_t td_warps = (int64_t)sm_count() * g->td_blocks_per_sm * (kBlock / 32);
        bool filled = !fuse_init;  // outputs of unreached vertices hold -1
        bool level_direct = !lpass;  // the layers store levels themselves
        int32_t *lvl = level_direct ? level : nullptr;
        auto fill_outputs = [&]() -> bfs_status {
            GB_LAUNCH(out_fill_kernel, grid_cap(n, kBlock, 8), kBlock, 0, st, n, root, g->visited,
                      g->base_vis, lvl, parent);
            filled = true;
            return BFS_OK;
        };
        for (int d = d_first; n_f > 0; ++d) {
            if (d > n) {  // a BFS has at most n layers: the counters are inconsistent
                set_error("bfs_run: internal error, traversal did not terminate after %lld layers",
                          (long long)n);
                cudaStreamSynchronize(st);
                return BFS_ERR_INTERNAL;
            }
            if (!level_direct && d + 1 >= kLevelRing) {
                // the next frontier would reuse slot 0: write the levels of
                // layers 0..d now and let the layers store theirs from here
                GB_LAUNCH(level_pass_kernel, grid_cap(g->nw_pad, kBlock / 32 * 8, 8), kBlock, 0, st,
                          g->ring, g->nw_pad, d + 1, n, level);
                level_direct = true;
                lvl = level;
            }
            if (hybrid && !decide(cfg, cur_bu, d, n, n_f, m_f, n_u, m_u)) {
                // a top-down layer: the device runs it and the ones after it
                // up to the next bottom-up decision (or the end)
                LoopState s1;
                s1.d = d;
                s1.n_f = n_f;
                s1.m_f = m_f;
                s1.n_u = n_u;
                s1.m_u = m_u;
                s1.degsum = degree_sum;
                s1.cur_bu = cur_bu;
                s1.have_queue = have_queue ? 1 : 0;
                const bfs_status ss = run_device_segment(g, level, parent, st, s1, true);
                if (ss != BFS_OK) return ss;
                adopt(s1);
                d = d_first - 1;  // the loop resumes at the layer the stretch stopped at
                continue;
            }
            cur_bu = decide(cfg, cur_bu, d, n, n_f, m_f, n_u, m_u);
            bfs_layer_stats ls;
            memset(&ls, 0, sizeof ls);
            ls.direction = cur_bu;
            ls.n_f = n_f;
            ls.m_f = m_f;
            ls.n_u = n_u;
            ls.m_u = m_u;
            degree_sum += m_f;
            int64_t *slot_cur = g->trace + (d % kRing) * kFields;
            int64_t *slot_next = g->trace + ((d + 1) % kRing) * kFields;
            int64_t *slot_zero = g->trace + ((d + 2) % kRing) * kFields;
            const size_t e0 = (size_t)d * 4;
            if (all_events) GB_CK(cudaEventRecord(event(e0), st));
            if (!cur_bu) {
                if (!have_queue) {
                    GB_LAUNCH(b2q_kernel, grid_cap(g->nw, kBlock * 4, 8), kBlock, 0, st, front, g->nw,
                              q_cur, (unsigned long long *)(slot_cur + T_CONV));
                    ls.converted = 1;
                }
                GB_CK(cudaMemsetAsync(next, 0, (size_t)g->nw_pad * 4, st));
                // Queue output only while the layer is small enough that one
                // atomicAdd per warp and round on the queue tail does not
                // serialise; a large layer leaves only the next bitmap, and the
                // queue is rebuilt by b2q if the next layer is top-down too.
                const int queue_mode = m_f <= kQueueModeMaxEdges ? 1 : 0;
                const int defer = td_defer(queue_mode, n_u - g->deg0, g->nw);
                TdArgs a{g->off, g->idx, g->visited, next, parent, lvl, q_next,
                         (unsigned long long *)(slot_next + T_NF), d + 1, queue_mode, cfg.td_claim,
                         defer};
                // Entries per warp so that a small frontier still covers the GPU,
                // and the grid-spread threshold at the frontier's edges per warp.
                const int per_warp = (int)std::min<int64_t>(32, std::max<int64_t>(1, (n_f + td_warps - 1) / td_warps));
                const int64_t grid_deg = std::min<int64_t>(
                    cfg.td_grid_degree,
                    std::max<int64_t>(4 * (int64_t)cfg.td_warp_degree, m_f / td_warps));
                const int td_grid = grid_cap((n_f + per_warp - 1) / per_warp, kBlock / 32,
                                             g->td_blocks_per_sm);
                if (all_events) GB_CK(cudaEventRecord(event(e0 + 1), st));
                GB_LAUNCH(td_kernel, td_grid, kBlock, 0, st, a, q_cur, n_f, per_warp, g->big,
                          (unsigned long long *)(slot_cur + T_BIG),
                          (unsigned long long *)(slot_next + T_MF), cfg.td_warp_degree, grid_deg,
                          slot_zero);
                if (m_f >= grid_deg) {
                    const int big_grid = (int)std::max<int64_t>(
                        1, std::min<int64_t>(m_f / 4096 + 1, (int64_t)sm_count() * g->td_blocks_per_sm));
                    GB_LAUNCH(td_big_kernel, big_grid, kBlock, 0, st, a, g->big,
                              (const unsigned long long *)(slot_cur + T_BIG),
                              (unsigned long long *)(slot_next + T_MF));
                }
                if (defer)
                    GB_LAUNCH(td_post_kernel, grid_cap(g->nw, kBlock, 8), kBlock, 0, st,
                              g->off, next, g->nw, lvl, d + 1,
                              (unsigned long long *)(slot_next + T_NF),
                              (unsigned long long *)(slot_next + T_MF));
                have_queue = queue_mode != 0;
            } else {
                if (all_events) GB_CK(cudaEventRecord(event(e0 + 1), st));
                // vertices still to find: unvisited and of degree > 0
                const int64_t active = n_u - g->deg0;
                if (cfg.bu_list_percent > 0 && active * 100 <= (int64_t)cfg.bu_list_percent * n) {
                    // sparse layer: a compacted list of them, one lane each
                    ls.converted = 2;
                    if (!filled) {
                        const bfs_status fs = fill_outputs();
                        if (fs != BFS_OK) return fs;
                    }
                    GB_CK(cudaMemsetAsync(next, 0, (size_t)g->nw_pad * 4, st));
                    GB_LAUNCH(bits_list_kernel, grid_cap(g->nw, kBlock * 4, 8), kBlock, 0, st,
                              g->visited, ~0u, g->nw, q_next,
                              (unsigned long long *)(slot_cur + T_ULIST));
                    GB_LAUNCH(bu_list_kernel,
                              grid_cap((active + 31) / 32, kBlock / 32, g->bu_list_blocks_per_sm),
                              kBlock, 0, st, g->off, g->idx, cfg.bu_head ? g->head : nullptr,
                              hskip, q_next, (const unsigned long long *)(slot_cur + T_ULIST),
                              g->visited, front, next, parent, lvl, d + 1, cfg.bu_probe,
                              (unsigned long long *)slot_next, slot_zero, 0);
                } else if (two_pass) {
                    // two passes: hub probes over the words, then the rows of
                    // the vertices whose hub missed, one lane each
                    ls.converted = 3;
                    const bool stream = cfg.hub_stream_stages > 0 &&
                                        active * 100 >= (int64_t)cfg.hub_stream_percent * n;
                    if (timing && !all_events) GB_CK(cudaEventRecord(event(e0 + 1), st));
                    if (stream) {
                        GB_LAUNCH(hub_stream_fn(cfg.hub_stream_stages, !filled),
                                  grid_cap(g->nw_pad / kWarpTile, kBlock / 32, g->hub_stream_occ),
                                  kBlock, hub_stream_smem_bytes(cfg.hub_stream_stages), st,
                                  g->hubc, g->wrank, g->wmeta, g->nw_pad, g->visited, front, next,
                                  g->pend, parent, lvl, d + 1, (unsigned long long *)slot_next,
                                  slot_zero, n, root);
                    } else {
                        GB_LAUNCH(bu_hubc_kernel,
                                  grid_cap(g->nw_pad, kBlock / 32 * 8, g->hubc_blocks_per_sm),
                                  kBlock, 0, st, g->hubc, g->wrank, g->nw_pad, g->visited, front,
                                  next, g->pend, parent, lvl, d + 1,
                                  (unsigned long long *)slot_next, slot_zero, filled ? 0 : 1,
                                  g->base_vis, n, root);
                    }
                    filled = true;
                    if (timing) GB_CK(cudaEventRecord(event(e0 + 3), st));
                    GB_LAUNCH(bits_list_kernel, grid_cap(g->nw, kBlock * 4, 8), kBlock, 0, st,
                              g->pend, 0u, g->nw, q_next,
                              (unsigned long long *)(slot_cur + T_ULIST));
                    GB_LAUNCH(bu_list_kernel,
                              grid_cap((active + 31) / 32, kBlock / 32, g->bu_list_blocks_per_sm),
                              kBlock, 0, st, g->off, g->idx, nullptr, 0, q_next,
                              (const unsigned long long *)(slot_cur + T_ULIST), g->visited, front,
                              next, parent, lvl, d + 1, cfg.bu_probe,
                              (unsigned long long *)slot_next, slot_zero, 1);
                } else {
                    if (!filled) {
                        const bfs_status fs = fill_outputs();
                        if (fs != BFS_OK) return fs;
                    }
                    decltype(BU1) const kernels[6] = {BU1, BU2, BU4, BU1H, BU2H, BU4H};
                    auto bu = kernels[bsel];
                    GB_LAUNCH(bu, bu_grid, kBlock, 0, st, g->off, g->idx, g->head, g->nw_pad,
                              g->visited, front, next, parent, lvl, d + 1, cfg.bu_probe,
                              (unsigned long long *)slot_next, slot_zero, bu_span_w, hskip);
                }
                have_queue = false;
            }
            if (all_events) GB_CK(cudaEventRecord(event(e0 + 2), st));
            {
                const bfs_status ps = publish_and_wait(g, slot_next, st);
                if (ps != BFS_OK) return ps;
            }
            if (g->h_slot[T_ERR]) {
                set_error("bfs_run: a bounded wait for a bulk copy ran out in layer %d", d);
                GB_CK(cudaStreamSynchronize(st));
                return BFS_ERR_TIMEOUT;
            }
            const int64_t found = g->h_slot[T_NF];
            // after a two-pass layer T_MF holds e_u after the layer (the
            // degree sum of the vertices still unvisited): e_f = e_u - that
            const int64_t m_new =
                (ls.converted == 3 && cur_bu) ? m_u - g->h_slot[T_MF] : g->h_slot[T_MF];
            ls.examined = cur_bu ? g->h_slot[T_EXAM] : m_f;
            ls.found = found;
            if (ls.converted == 3 && cur_bu) ls.hub_found = g->h_slot[T_HUB];
            g->last.push_back(ls);
            n_u -= found;
            m_u -= m_new;
            n_f = found;
            m_f = m_new;
            if (lpass) {
                front = next;
                next = g->ring + (int64_t)((d + 2) % kLevelRing) * g->nw_pad;
            } else {
                std::swap(front, next);
            }
            std::swap(q_cur, q_next);
        }
        if (!filled) {
            const bfs_status fs = fill_outputs();
            if (fs != BFS_OK) return fs;
        }
        if (!level_direct) {
            // slot j of the ring holds level j, for every layer run
            const int slots = (int)std::min<size_t>(g->last.size() + 1, kLevelRing);
            GB_LAUNCH(level_pass_kernel, grid_cap(g->nw_pad, kBlock / 32 * 8, 8), kBlock, 0, st,
                      g->ring, g->nw_pad, slots, n, level);
        }
        GB_CK(cudaStreamSynchronize(st));  // outputs complete, late errors surface
        g->last_component_edges = degree_sum / 2;
        if (timing) {
            for (size_t d = 0; d < g->last.size(); ++d) {
                float t0 = 0, t1 = 0, t2 = 0;
                if (all_events) {
                    cudaEventElapsedTime(&t0, g->events[4 * d], g->events[4 * d + 2]);
                    cudaEventElapsedTime(&t1, g->events[4 * d + 1], g->events[4 * d + 2]);
                }
                if (g->last[d].direction == 1 && g->last[d].converted == 3)
                    cudaEventElapsedTime(&t2, g->events[4 * d + 1], g->events[4 * d + 3]);
                g->last[d].ms_total = t0;
                g->last[d].ms_main = t1;
                g->last[d].ms_sweep = t2;
            }
        }
    }
    if (cfg.parent_min) {
        GB_LAUNCH(min_parent_kernel, grid_cap(n, kBlock, 8), kBlock, 0, st, g->off, g->idx,
                  level, parent, n, root, g->rows_sorted);
        if (!host_out) GB_CK(cudaStreamSynchronize(st));
    }
    if (async_out) {
        // the copy stream takes the results after the traversal; the next
        // traversal (other output pair) overlaps it
        GB_CK(cudaEventRecord(g->hout_ready, st));
        GB_CK(cudaStreamWaitEvent(g->copy_st, g->hout_ready, 0));
        GB_CK(cudaMemcpyAsync(level_out, level, (size_t)n * 4, cudaMemcpyDeviceToHost, g->copy_st));
        if (parent_out)
            GB_CK(cudaMemcpyAsync(parent_out, parent, (size_t)n * 4, cudaMemcpyDeviceToHost,
                                  g->copy_st));
        GB_CK(cudaEventRecord(g->hout_done[slot], g->copy_st));
    } else if (host_out) {
        GB_CK(cudaMemcpyAsync(level_out, level, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
        if (parent_out)
            GB_CK(cudaMemcpyAsync(parent_out, parent, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
        GB_CK(cudaStreamSynchronize(st));
    }
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_graph_sync(bfs_graph *g) {
    clear_error();
    if (!g) {
        set_error("bfs_graph_sync: null graph");
        return BFS_ERR_INVALID;
    }
    if (g->copy_st) GB_CK(cudaStreamSynchronize(g->copy_st));
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_last_run_stats(const bfs_graph *g, bfs_layer_stats *out,
                                                 int32_t cap, int32_t *layers,
                                                 int64_t *component_edges) {
    clear_error();
    if (!g || cap < 0 || (cap > 0 && !out)) {
        set_error("bfs_last_run_stats: null graph or output");
        return BFS_ERR_INVALID;
    }
    const int32_t L = (int32_t)g->last.size();
    for (int32_t i = 0; i < std::min(cap, L); ++i) out[i] = g->last[i];
    if (layers) *layers = L;
    if (component_edges) *component_edges = g->last_component_edges;
    return BFS_OK;
}

// ---------------------------------------------------------------------------
// bfs_run_noalloc: the same traversal with its scratch in a fixed device array
// instead of graph-owned allocations, for callers that may not allocate.
// ---------------------------------------------------------------------------
namespace gbfs {
namespace {

constexpr int64_t kNoAllocMaxN = 1 << 20;
constexpr int64_t kNoAllocNwPad = ((((kNoAllocMaxN + 31) / 32) + 31) / 32) * 32;
constexpr size_t kNoAllocBitmapBytes = (size_t)kNoAllocNwPad * 4;
constexpr size_t kNoAllocQueueBytes = (size_t)kNoAllocMaxN * 4;
constexpr size_t kNoAllocTraceBytes = (size_t)kRing * kFields * 8;
// visited, base, front, next | q_a, q_b, big | trace
constexpr size_t kNoAllocBytes =
    4 * kNoAllocBitmapBytes + 3 * kNoAllocQueueBytes + kNoAllocTraceBytes;

// Shared by every call in the process, one copy per device that loads the
// library (about 12.5 MiB), kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch, looked up once per device with that
// device current (the host-side symbol is only a stand-in).
bfs_status noalloc_scratch(unsigned char **out) {
    static std::mutex mu;
    static std::vector<unsigned char *> addr;
    int dev = 0;
    GB_CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void *p = nullptr;
        GB_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        addr[dev] = (unsigned char *)p;
    }
    *out = addr[dev];
    return BFS_OK;
}

}  // namespace
}  // namespace gbfs

extern "C" BFS_API bfs_status bfs_run_noalloc(const int64_t *offsets, const int32_t *indices,
                                              int64_t n, int64_t nnz, int32_t root,
                                              int32_t *level_out, int32_t *parent_out,
                                              void *stream) {
    clear_error();
    if (!offsets || (nnz > 0 && !indices) || !level_out || !parent_out || nnz < 0 || n < 1) {
        set_error("bfs_run_noalloc: need device offsets/indices/level_out/parent_out and n >= 1");
        return BFS_ERR_INVALID;
    }
    if (n > kNoAllocMaxN) {
        set_error("bfs_run_noalloc: n = %lld exceeds the fixed scratch limit of %lld vertices",
                  (long long)n, (long long)kNoAllocMaxN);
        return BFS_ERR_INVALID;
    }
    if (root < 0 || root >= n) {
        set_error("bfs_run_noalloc: root out of range");
        return BFS_ERR_INVALID;
    }
    cudaStream_t st = as_stream(stream);
    {
        // e_u starts from nnz (Sec. 4): a count that disagrees with the CSR
        // would skew every direction decision, so it is checked before any
        // launch (one 8-byte read of offsets[n])
        int64_t last = -1;
        GB_CK(cudaMemcpyAsync(&last, offsets + n, sizeof last, cudaMemcpyDeviceToHost, st));
        GB_CK(cudaStreamSynchronize(st));
        if (last != nnz) {
            set_error("bfs_run_noalloc: nnz = %lld but offsets[n] = %lld", (long long)nnz,
                      (long long)last);
            return BFS_ERR_INVALID;
        }
    }
    unsigned char *base = nullptr;
    bfs_status s = noalloc_scratch(&base);
    if (s != BFS_OK) return s;
    uint32_t *visited = (uint32_t *)base;
    uint32_t *base_vis = visited + kNoAllocNwPad;
    uint32_t *front = base_vis + kNoAllocNwPad;
    uint32_t *next = front + kNoAllocNwPad;
    int32_t *q_cur = (int32_t *)(next + kNoAllocNwPad);
    int32_t *q_next = q_cur + kNoAllocMaxN;
    int32_t *big = q_next + kNoAllocMaxN;
    int64_t *trace = (int64_t *)(big + kNoAllocMaxN);

    bfs_config cfg;
    bfs_config_default(&cfg);
    const int64_t nw = (n + 31) / 32;
    const int64_t nw_pad = ((nw + 31) / 32) * 32;
    int bu_occ = 1, td_occ = 1;
    GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bu_occ, BU2, kBlock, 0));
    GB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&td_occ, td_kernel, kBlock, 0));
    // bottom-up warp tasks sized to cover the machine, as in bfs_run's host loop
    const int64_t bu_full = (int64_t)sm_count() * std::max(1, bu_occ);
    const int span = bu_span(nw_pad >> 5, 2, bu_full * (kBlock / 32));
    const int bu_grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((nw_pad >> 5) * (32 / span) / (kBlock / 32) + 1, bu_full));
    const int64_t td_warps = (int64_t)sm_count() * td_occ * (kBlock / 32);

    // The traversal proper. On any error the stream is drained before the
    // status is returned, so no kernel of this call still writes the shared
    // array or the caller's outputs afterwards.
    auto traverse = [&]() -> bfs_status {
        // Every buffer the traversal reads before writing is set here: the
        // base and visited bitmaps, the frontier bitmap, the first queue entry
        // and the whole trace ring (init_kernel), so nothing of a previous
        // call leaks in.
        GB_LAUNCH(base_vis_kernel, grid_cap(nw_pad, kBlock, 8), kBlock, 0, st, offsets, n,
                  nw_pad, base_vis);
        GB_LAUNCH(init_kernel, grid_cap(std::max(n, nw_pad), kBlock, 8), kBlock, 0, st, n,
                  nw_pad, root, offsets, base_vis, nullptr, level_out, parent_out, visited,
                  front, q_cur, trace, 1);
        int64_t h[kFields];
        GB_CK(cudaMemcpyAsync(h, trace, sizeof h, cudaMemcpyDeviceToHost, st));
        GB_CK(cudaStreamSynchronize(st));
        int64_t n_f = 1, m_f = h[T_MF];
        int64_t n_u = n - 1, m_u = nnz - m_f;
        int cur_bu = 0;
        bool have_queue = true;
        for (int d = 0; n_f > 0; ++d) {
            if (d > n) {  // a BFS has at most n layers: the counters are inconsistent
                set_error("bfs_run_noalloc: internal error, traversal did not terminate "
                          "after %lld layers",
                          (long long)n);
                return BFS_ERR_INTERNAL;
            }
            cur_bu = decide(cfg, cur_bu, d, n, n_f, m_f, n_u, m_u);
            int64_t *slot_cur = trace + (d % kRing) * kFields;
            int64_t *slot_next = trace + ((d + 1) % kRing) * kFields;
            int64_t *slot_zero = trace + ((d + 2) % kRing) * kFields;
            if (!cur_bu) {
                if (!have_queue)
                    GB_LAUNCH(b2q_kernel, grid_cap(nw, kBlock * 4, 8), kBlock, 0, st, front, nw,
                              q_cur, (unsigned long long *)(slot_cur + T_CONV));
                GB_CK(cudaMemsetAsync(next, 0, (size_t)nw_pad * 4, st));
                const int queue_mode = m_f <= kQueueModeMaxEdges ? 1 : 0;
                const int defer = td_defer(queue_mode, n_u, nw);
                TdArgs a{offsets, indices, visited, next, parent_out, level_out, q_next,
                         (unsigned long long *)(slot_next + T_NF), d + 1, queue_mode,
                         cfg.td_claim, defer};
                const int per_warp = (int)std::min<int64_t>(
                    32, std::max<int64_t>(1, (n_f + td_warps - 1) / td_warps));
                const int64_t grid_deg = std::min<int64_t>(
                    cfg.td_grid_degree,
                    std::max<int64_t>(4 * (int64_t)cfg.td_warp_degree, m_f / td_warps));
                GB_LAUNCH(td_kernel, grid_cap((n_f + per_warp - 1) / per_warp, kBlock / 32, td_occ),
                          kBlock, 0, st, a, q_cur, n_f, per_warp, big,
                          (unsigned long long *)(slot_cur + T_BIG),
                          (unsigned long long *)(slot_next + T_MF), cfg.td_warp_degree, grid_deg,
                          slot_zero);
                if (m_f >= grid_deg)
                    GB_LAUNCH(td_big_kernel,
                              (int)std::max<int64_t>(
                                  1, std::min<int64_t>(m_f / 4096 + 1, (int64_t)sm_count() * td_occ)),
                              kBlock, 0, st, a, big, (const unsigned long long *)(slot_cur + T_BIG),
                              (unsigned long long *)(slot_next + T_MF));
                if (defer)
                    GB_LAUNCH(td_post_kernel, grid_cap(nw, kBlock / 4, 8), kBlock, 0, st, offsets,
                              next, nw, level_out, d + 1, (unsigned long long *)(slot_next + T_NF),
                              (unsigned long long *)(slot_next + T_MF));
                have_queue = queue_mode != 0;
            } else {
                GB_LAUNCH(BU2, bu_grid, kBlock, 0, st, offsets, indices, nullptr, nw_pad, visited,
                          front, next, parent_out, level_out, d + 1, cfg.bu_probe,
                          (unsigned long long *)slot_next, slot_zero, span, 0);
                have_queue = false;
            }
            GB_CK(cudaMemcpyAsync(h, slot_next, sizeof h, cudaMemcpyDeviceToHost, st));
            GB_CK(cudaStreamSynchronize(st));
            n_u -= h[T_NF];
            m_u -= h[T_MF];
            n_f = h[T_NF];
            m_f = h[T_MF];
            std::swap(front, next);
            std::swap(q_cur, q_next);
        }
        return BFS_OK;
    };
    s = traverse();
    if (s != BFS_OK) cudaStreamSynchronize(st);  // its own error, if any, is already recorded
    return s;
}
