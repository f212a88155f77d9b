// graph.cuh -- the bfs_graph object shared by the single-source and the
// batched traversal, and small host helpers used by both.
#pragma once

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace gbfs {

constexpr int kRing = 64;  // trace ring slots (layers)
constexpr int kFields = 8;
enum TraceField {
    T_NF = 0, T_MF = 1, T_EXAM = 2, T_CONV = 3, T_BIG = 4, T_ULIST = 5, T_HUB = 6,
    T_ERR = 7  // set by a kernel whose bounded wait ran out
};
constexpr int kBlock = 256;
constexpr int kBigBatch = 1024;
constexpr int64_t kQueueModeMaxEdges = 1 << 18;
constexpr int kTdK = 4;  // edges per lane in flight in the warp and grid top-down paths
constexpr int kLevelRing = 16;  // frontier bitmaps kept for the level pass

}  // namespace gbfs

struct MsState;  // batched-traversal buffers (msbfs.cu), allocated on first use

struct bfs_graph {
    int device = 0;
    int64_t n = 0, nnz = 0, nw = 0, nw_pad = 0;
    const int64_t *off = nullptr;
    const int32_t *idx = nullptr;
    int64_t *off_own = nullptr;
    int32_t *idx_own = nullptr;
    uint32_t *visited = nullptr, *bm_a = nullptr, *bm_b = nullptr;
    uint32_t *pend = nullptr;      // vertices whose hub missed (two-pass bottom-up)
    int rows_sorted = -1;          // every CSR row ascending: -1 not checked yet
    int bu_hub_blocks_per_sm = 0;
    int hubc_blocks_per_sm = 1;    // resident blocks per SM of the compact gather sweep
    int hub_stream_occ = 0;        // resident blocks per SM of the streaming sweep
    int hub_stream_occ_stages = 0; // ... for this stage count (0 = not queried)
    int2 *head = nullptr;          // {first probe (-1 if none), degree}
    // compact hub records of the degree >= 1 vertices, in id order: hub id,
    // bit 31 set when the vertex has degree 1; wrank[w] = degree >= 1
    // vertices before bitmap word w (nw_pad + 1 entries)
    uint32_t *hubc = nullptr, *wrank = nullptr;
    uint2 *wmeta = nullptr;        // {base word, wrank} per word, for the streaming sweep
    int64_t n1 = 0;                // vertices of degree >= 1
    int head_kind = 0;             // what head holds: 1 first neighbour, 2 hub
    uint32_t *comp_in = nullptr;   // vertices in the component of comp_rep
    int32_t comp_rep = -1;         // highest-degree vertex; -1 = not built yet
    int64_t deg0 = 0;              // vertices of degree 0
    uint32_t *base_vis = nullptr;  // bits that start every traversal visited:
                                   // degree-0 vertices and ids past n
    int32_t *q_a = nullptr, *q_b = nullptr, *big = nullptr;
    // level pass: kLevelRing frontier bitmaps of nw_pad words (slot j holds
    // the vertices of level j), allocated on first use
    uint32_t *ring = nullptr;
    int32_t *parent_scratch = nullptr, *level_scratch = nullptr;
    // host_async: two device output pairs used in turn, copied to the host on
    // copy_st; hout_done[i] marks the end of pair i's copy
    int32_t *hout_level[2] = {nullptr, nullptr}, *hout_parent[2] = {nullptr, nullptr};
    cudaEvent_t hout_done[2] = {nullptr, nullptr}, hout_ready = nullptr;
    cudaStream_t copy_st = nullptr;
    int hout_turn = 0;
    int64_t *trace = nullptr;
    int64_t *misc = nullptr;    // 8 device words for one-off flags and maxima
    int64_t *h_slot = nullptr;  // pinned, kFields entries
    // mapped pinned block the host loop polls: kFields counters then a
    // sequence number, written by publish_kernel (d_pub = device address)
    int64_t *h_pub = nullptr, *d_pub = nullptr;
    int64_t pub_seq = 0;
    bfs_config cfg;
    std::vector<bfs_layer_stats> last;
    int64_t last_component_edges = 0;
    std::vector<cudaEvent_t> events;
    int bu_blocks_per_sm[6] = {1, 1, 1, 1, 1, 1};  // BU1, BU2, BU4, BU1H, BU2H, BU4H
    int td_blocks_per_sm = 1;
    int bu_list_blocks_per_sm = 1;
    int persist_blocks_per_sm = 0;  // device-loop kernel, 0 = not queried yet
    int64_t *pctl = nullptr, *h_pctl = nullptr;  // device-loop layer records
    // graph loop (device_loop = 3): instantiated graph, its device state and
    // records (gl_mem), their pinned host copy, and the kernels' fixed
    // arguments (host heap); built on first use, dropped on a config change
    cudaGraph_t gl_graph = nullptr;
    cudaGraphExec_t gl_exec = nullptr;
    void *gl_mem = nullptr, *h_gl = nullptr, *gl_static = nullptr;
    MsState *ms = nullptr;
};

namespace gbfs {

inline int grid_cap(int64_t work_items, int per_block, int blocks_per_sm) {
    int64_t g = (work_items + per_block - 1) / per_block;
    const int64_t cap = (int64_t)sm_count() * std::max(1, blocks_per_sm);
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

void free_ms_state(bfs_graph *g);  // msbfs.cu

}  // namespace gbfs
