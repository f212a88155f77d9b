/*
 * bfs.h -- C ABI of the GB300 hybrid breadth-first-search library.
 *
 * The library implements the hybrid BFS of Paredes, Riley and Lujan,
 * "Vectorization of Hybrid Breadth First Search on the Intel Xeon Phi":
 * a layer-synchronous traversal (Sec. 4) that runs each layer either as the
 * top-down step of Alg. 1 or as the bottom-up step of Alg. 2 / Sec. 5, the
 * direction being chosen per layer by the switch of Alg. 3. Every step runs in
 * this library's own CUDA kernels for sm_103a on one GPU.
 *
 * Conventions shared by every entry point
 *   - Every call returns a bfs_status. Nothing aborts, nothing traps; on an
 *     error bfs_last_error() returns a message for the calling thread.
 *   - Arguments are checked on the host before any launch: null pointers,
 *     sizes out of range and roots outside [0, n) give BFS_ERR_INVALID.
 *   - Vertex ids are int32 in [0, n), n < 2^31. CSR offsets are int64
 *     (n + 1 entries, offsets[0] = 0, offsets[n] = nnz); CSR indices are
 *     int32 (nnz entries). The graph must be symmetric: the bottom-up step
 *     reads Adj[v] as the in-edges of v (Sec. 6.2, edges are bidirectional).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Device pointers must belong to the current CUDA device.
 *   - Output encoding (Sec. 4, the predecessor list P): level[v] is the hop
 *     distance from the root, -1 when unreachable; parent[root] = root,
 *     parent[v] = -1 when unreachable.
 *   - A bfs_graph is not thread-safe: one call at a time per graph.
 */
#ifndef GB300_HYBRID_BFS_H
#define GB300_HYBRID_BFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define BFS_API __attribute__((visibility("default")))
#else
#define BFS_API
#endif

typedef enum bfs_status {
    BFS_OK = 0,
    BFS_ERR_INVALID = 1,   /* bad argument; nothing was launched            */
    BFS_ERR_OOM = 2,       /* a device or pinned allocation failed          */
    BFS_ERR_CUDA = 3,      /* a CUDA call failed; see bfs_last_error()      */
    BFS_ERR_TIMEOUT = 4,   /* a bounded device-side wait ran out            */
    BFS_ERR_DEPTH = 5,     /* an int8 level would exceed 127                */
    BFS_ERR_BUSY = 6,      /* the server has no room for the request        */
    BFS_ERR_SHUTDOWN = 7,  /* the server is shutting down                   */
    BFS_ERR_INTERNAL = 8   /* the library's own consistency check failed   */
} bfs_status;

/* Message for the last failed call made by this thread ("" if none). */
BFS_API const char *bfs_last_error(void);

/* Number of kernels this library has launched in this process so far. */
BFS_API int64_t bfs_launch_count(void);

/* ---------------------------------------------------------------------- */
/* Graph generation (Sec. 6.2: Graph500 Kronecker graphs built on the      */
/* R-MAT model with initiator A, B, C, D).                                 */
/* ---------------------------------------------------------------------- */
#define BFS_GEN_RMAT 0   /* R-MAT / Kronecker, initiator (a, b, c, 1-a-b-c) */
#define BFS_GEN_ER 1     /* Erdos-Renyi control: uniform endpoints          */

/* Writes the m = edgefactor * 2^scale generated edges (src[e], dst[e]) into
 * caller-owned device arrays of m int32 each. scale in [1, 30].
 * Edge e at bit level b draws the high 32 bits of SplitMix64 output
 * e*scale + b of `seed` and picks a quadrant by comparing them with
 * floor(a*2^32), floor((a+b)*2^32), floor((a+b+c)*2^32); the bits are then
 * relabelled by a seeded bijection of [0, 2^scale). The ER control uses the
 * top `scale` bits of outputs 2e and 2e+1. Stream-ordered; returns at once. */
BFS_API bfs_status bfs_generate_edges(int32_t kind, int32_t scale, int32_t edgefactor,
                                      uint64_t seed, double a, double b, double c,
                                      int32_t *src, int32_t *dst, void *stream);

/* Symmetric CSR from an edge list (Sec. 6.2: each edge is stored in both
 * directions; Sec. 6.3: CSR). Self-loops are dropped, every row is sorted
 * ascending and duplicates are removed.
 *   src, dst    device, m int32 each, endpoints in [0, n)
 *   offsets     device, caller-owned, n + 1 int64 (written)
 *   indices     device, caller-owned, room for 2*m int32 (first nnz written)
 *   nnz_out     host, receives nnz
 * Temporary device memory (about 16*m bytes) is taken with cudaMallocAsync
 * on `stream` and released before return. Synchronises `stream`.
 * An endpoint outside [0, n) gives BFS_ERR_INVALID. */
BFS_API bfs_status bfs_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                 int64_t *offsets, int32_t *indices, int64_t *nnz_out,
                                 void *stream);

/* Seeded distinct roots of degree >= 1 (Sec. 6.3: 64 BFS executions from
 * random starting vertices; degree-0 roots would report zero TEPS).
 * Candidate j = SplitMix64 output j of `seed` modulo n; candidates are taken
 * in order, skipping degree-0 vertices and repeats, until k are chosen or
 * max_draws candidates were seen.
 *   offsets     device, n + 1 int64
 *   roots_out   device, k int32 (first *count_out written)
 *   count_out   host, number of roots chosen (may be < k)
 * k in [1, 4096]. Synchronises `stream`. */
BFS_API bfs_status bfs_sample_roots(const int64_t *offsets, int64_t n, uint64_t seed, int32_t k,
                                    int64_t max_draws, int32_t *roots_out, int32_t *count_out,
                                    void *stream);

/* ---------------------------------------------------------------------- */
/* Graphs and the single-source hybrid BFS (Alg. 1-3, Sec. 5).             */
/* ---------------------------------------------------------------------- */
typedef struct bfs_graph bfs_graph;

/* Direction policies for Alg. 3 (tests hold hysteresis: in top-down mode
 * switch to bottom-up iff the f test passes; in bottom-up mode switch back
 * iff the g test passes; layer 0 starts top-down).                        */
#define BFS_POLICY_EDGE 0    /* f: e_f > e_u / alpha ; g: v_f < n / beta       */
#define BFS_POLICY_VERTEX 1  /* f: v_f > n_u >> 10   ; g: v_f < n >> 6 (Table 2)*/
#define BFS_POLICY_FORCED 2  /* layer d runs forced[min(d, forced_len-1)]      */

typedef struct bfs_config {
    int32_t policy;          /* BFS_POLICY_*                                  */
    int32_t forced_len;      /* 1..64 entries used by BFS_POLICY_FORCED       */
    uint8_t forced[64];      /* 0 = top-down, 1 = bottom-up                   */
    double alpha;            /* edge policy, top-down -> bottom-up            */
    double beta;             /* edge policy, bottom-up -> top-down            */
    int32_t bu_probe;        /* neighbours a thread tests on its own in the
                                bottom-up step before the warp-cooperative
                                scan takes over (the MAX_POS of Sec. 5.2);
                                1..64                                          */
    int32_t td_warp_degree;  /* top-down: degree from which one warp expands
                                a vertex (smaller ones share a warp)           */
    int32_t td_grid_degree;  /* top-down: largest degree threshold above which
                                a vertex's edges are spread over the whole
                                grid (the threshold used per layer is the
                                frontier's edges per resident warp, clamped to
                                [4*td_warp_degree, td_grid_degree])            */
    int32_t timing;          /* 1 = record CUDA events around each layer
                                (ms_total, ms_main, ms_sweep); 2 = only around
                                each hub sweep (ms_sweep), so fewer event
                                records delay the next layer's launches      */
    int32_t bu_words;        /* bottom-up: bitmap words a warp keeps in
                                flight (1, 2 or 4)                             */
    int32_t td_claim;        /* top-down claim of a vertex: 0 = atomicCAS on
                                parent[v] (-1 -> u); 1 (default) = atomicOr
                                on the visited bitmap word, then plain parent
                                store. With 1, the host loop and two-pass
                                bottom-up layers, the -1 fill of level and
                                parent is done by the first bottom-up sweep
                                instead of before the traversal             */
    int32_t bu_head;         /* the bottom-up step first tests the neighbour
                                held in an 8-byte record per vertex
                                {neighbour, degree}, built on first use (8*n
                                bytes): one coalesced load instead of a
                                row-bound pair and a random index sector.
                                1 = the row's first entry (the scan then goes
                                on from its second); 2 = the hub, the
                                neighbour of largest degree (smallest id on
                                ties), the likeliest to be in an early
                                frontier (on a miss the row is scanned from
                                its first entry; Alg. 2 accepts any frontier
                                neighbour, so levels are unchanged and the
                                parent is the hub whenever it is in the
                                frontier). With 2, graphs with at least 8
                                bitmap words per resident warp run each dense
                                bottom-up layer in two passes: a sweep that
                                tests every unvisited vertex's hub, then a
                                row scan of the compacted hub misses, one
                                thread each (n/8 more bytes); smaller graphs
                                test the hub inside the one-pass scan.
                                0 = read the CSR only                        */
    int32_t prune_components;/* 1 = vertices outside the root's connected
                                component start as visited, so bottom-up
                                layers skip them (results unchanged; only the
                                edges-examined count shrinks). The component
                                of the highest-degree vertex is found once, by
                                one traversal on first use, and kept (n/8
                                bytes); roots outside it are not pruned.
                                Off by default: on R-MAT graphs almost every
                                vertex outside the giant component has degree
                                0 and is skipped anyway                       */
    int32_t bu_list_percent; /* bottom-up layers with at most this percentage
                                of n vertices left to find (unvisited, degree
                                > 0) run on a compacted list of those vertices,
                                one thread each, instead of one warp per
                                bitmap word; 0 = never                        */
    int32_t device_loop;     /* 1 = run all layers in one cooperative launch
                                whose blocks take the Alg. 3 decision on the
                                device, between bounded grid barriers (no host
                                round trip per layer; per-layer times are not
                                recorded); 0 = host loop; 2 (default) = the
                                device loop for n <= 2^25, where the host round
                                trips weigh most, the host loop above;
                                3 = graph loop: the host loop's kernels as one
                                CUDA graph (a WHILE node over a SWITCH node)
                                whose one-thread step kernel takes the Alg. 3
                                decision on the device between layers; built
                                on first use per configuration (at most 256
                                layers per graph launch, relaunched until the
                                traversal ends); with timing = 1 the host
                                loop runs instead; 4 = hybrid: each stretch
                                of top-down layers runs in one cooperative
                                launch of the device loop (which returns at
                                the first bottom-up decision), the bottom-up
                                layers from the host (timing = 1: the host
                                loop throughout)                              */
    int32_t host_async;      /* with host output buffers: 1 = bfs_run returns
                                once the traversal is done and the copy of its
                                results to the host runs on the graph's own
                                copy stream, overlapping the next traversal;
                                the buffers are complete after bfs_graph_sync
                                (two calls' copies may be in flight; the
                                outputs of a call must stay untouched until
                                then). 0 (default) = bfs_run returns with the
                                copy done                                      */
    int32_t parent_min;      /* 1 = after the traversal each reached vertex's
                                parent becomes its smallest-id neighbour one
                                level up: one deterministic tree among the
                                valid ones (Sec. 7.1), the same on every run
                                and equal to a sequential reference's.
                                Costs a pass over the reached vertices' rows
                                (early exit when every row is sorted ascending,
                                which is checked once): about 12.5 ms per BFS
                                on a scale-26 R-MAT graph, whose hubs one level
                                below few candidates scan long rows            */
    int32_t hub_stream_stages; /* two-pass bottom-up layers: the hub sweep of a
                                dense layer reads the head records of tiles of
                                1024 vertices through bulk copies into shared
                                memory, this many tiles in flight per block
                                (2, 3, 4, 6 or 8); 0 = never (every sweep
                                gathers the records of unvisited vertices).
                                Results are the same either way              */
    int32_t hub_stream_percent; /* a hub sweep streams when at least this
                                percentage of n vertices is still to find
                                (unvisited, degree > 0); 0..100              */
    int32_t level_pass;      /* host loop: 1 = the layers do not
                                store levels; each layer's frontier bitmap is
                                kept in a ring of 16 (2n bytes) and one pass
                                after the traversal writes every level as
                                whole rows, so the scattered 4-byte level
                                stores of later layers (and the sector fills
                                they cost) disappear; a traversal that reaches
                                layer 15 writes the levels so far and stores
                                the rest as found. 0 (default) = levels
                                stored as found                              */
} bfs_config;

/* Fills `cfg` with the defaults (edge policy, alpha 20, beta 200, hub head
 * records, bitmap claims, device loop up to 2^25 vertices, ...). */
BFS_API void bfs_config_default(bfs_config *cfg);

#define BFS_DEVICE_PTRS 1u  /* offsets / indices are device pointers           */
#define BFS_BORROW 2u       /* keep the caller's device arrays (no copy); they
                               must outlive the graph. Needs BFS_DEVICE_PTRS.  */
#define BFS_VALIDATE 4u     /* check offsets[0]=0, monotone offsets,
                               offsets[n]=nnz and indices in [0, n)            */
#define BFS_VALIDATE_SYMMETRIC 8u  /* also check, after the checks of
                               BFS_VALIDATE (implied), that every row is
                               strictly ascending and that every entry u of
                               row v has its reverse entry v in row u: the
                               bottom-up step reads a row as the vertex's
                               in-edges, so it needs the undirected graph of
                               Sec. 6.2 stored both ways. Costs a binary
                               search per entry (0.56 s at scale 26, 2.1 G
                               entries). Failure: BFS_ERR_INVALID          */

/* Creates a graph from a symmetric CSR (layout above) and allocates its
 * per-traversal scratch: five n-bit bitmaps (visited, frontier, next, the
 * degree-0 mask and the two-pass step's hub misses), three n-entry vertex
 * lists (two queues and the list of grid-spread vertices) and a small counter
 * block: about 12.6*n bytes. The 8-byte head records (cfg.bu_head, 8*n bytes)
 * are built here when cfg asks for them (the defaults do), else by the first
 * bfs_run that does; whatever else a configuration needs is allocated by
 * bfs_graph_reserve or, failing that, by the first bfs_run that needs it.
 * Without BFS_BORROW the CSR is copied into library memory and the caller may
 * free its arrays. cfg may be NULL (defaults). Synchronous. */
BFS_API bfs_status bfs_graph_create(const int64_t *offsets, const int32_t *indices, int64_t n,
                                    int64_t nnz, uint32_t flags, const bfs_config *cfg,
                                    bfs_graph **out);

/* Replaces the graph's configuration (cfg may be NULL for the defaults). */
BFS_API bfs_status bfs_graph_set_config(bfs_graph *g, const bfs_config *cfg);

/* Device pointers and sizes of the graph's CSR (library- or caller-owned). */
BFS_API bfs_status bfs_graph_info(const bfs_graph *g, const int64_t **offsets,
                                  const int32_t **indices, int64_t *n, int64_t *nnz);

/* Frees everything the graph owns. NULL is accepted. */
BFS_API bfs_status bfs_graph_destroy(bfs_graph *g);

/* Allocates and builds now, for the graph's current configuration, all
 * that bfs_run would otherwise allocate on first use: the head records of
 * the configured kind, the device-loop records or the graph loop's CUDA
 * graph (cfg.device_loop), the component mask (cfg.prune_components: one
 * traversal), the rows-sorted check (cfg.parent_min), and, per flags,
 *   BFS_RESERVE_HOST_OUT   scratch for host output buffers (cfg.host_async:
 *                          the two device output pairs and the copy stream)
 *   BFS_RESERVE_NO_PARENT  scratch for parent_out = NULL
 * After it, bfs_run calls with this configuration and those kinds of output
 * make no device or pinned-host allocation (bfs_alloc_count() stays put),
 * so no allocation, and no implicit synchronisation of one, lands inside a
 * latency-measured call. Changing the configuration may need another call.
 * Synchronous on `stream`. */
#define BFS_RESERVE_HOST_OUT 1u
#define BFS_RESERVE_NO_PARENT 2u
BFS_API bfs_status bfs_graph_reserve(bfs_graph *g, uint32_t flags, void *stream);

/* Number of device and pinned-host allocations this library has made in
 * this process so far (cudaMalloc, cudaMallocAsync, cudaHostAlloc), for
 * checking that a reserved or warmed-up path allocates nothing. */
BFS_API int64_t bfs_alloc_count(void);

/* Hybrid BFS from `root` (Alg. 3). level_out / parent_out are n int32 each,
 * caller-owned, either both device memory or both host memory (pageable or
 * pinned); parent_out may be NULL. With host buffers the results are copied
 * back before return (cfg.host_async: the copy may still run, see
 * bfs_graph_sync). Work is ordered on `stream`, and the direction of each
 * layer is chosen from the layer counters by the host (host loop) or on the
 * device (device and graph loops, cfg.device_loop); either way the call
 * returns after the traversal has finished. Parents found by a bottom-up
 * layer are the vertex's hub when it is in the frontier (bu_head = 2), else
 * the first frontier neighbour in CSR order (Alg. 2); parents found by a
 * top-down layer are whichever frontier neighbour claimed the vertex first
 * (any valid tree, Sec. 7.1); cfg.parent_min replaces them all by the
 * smallest-id neighbour one level up. */
BFS_API bfs_status bfs_run(bfs_graph *g, int32_t root, int32_t *level_out, int32_t *parent_out,
                           void *stream);

/* Waits for the host copies that bfs_run left in flight (cfg.host_async) and
 * returns the first error among them; BFS_OK when none is pending. */
BFS_API bfs_status bfs_graph_sync(bfs_graph *g);

/* Per-layer record of the last bfs_run on this graph. Layer d is the
 * frontier of the vertices at level d. Counters follow Sec. 4: v_f (n_f),
 * e_f (m_f), and the unvisited vertex / edge counts n_u, m_u.             */
typedef struct bfs_layer_stats {
    int32_t direction;  /* 0 = top-down, 1 = bottom-up                          */
    int32_t converted;  /* top-down: 1 = the frontier bitmap was turned into a
                           queue; bottom-up: 2 = the layer ran on the compacted
                           list of vertices still to find (bu_list_percent),
                           3 = it ran in two passes (hub sweep, then the row
                           scans of the hub misses; bu_head = 2)              */
    int64_t n_f;        /* vertices in the frontier                            */
    int64_t m_f;        /* sum of their degrees                                */
    int64_t n_u;        /* vertices not yet visited                            */
    int64_t m_u;        /* sum of their degrees                                */
    int64_t examined;   /* edges examined: all frontier edges top-down; up to
                           and including the first hit (or the whole row)
                           bottom-up                                           */
    int64_t found;      /* vertices of the next layer                          */
    float ms_total;     /* layer time, when cfg.timing = 1 (else 0)            */
    float ms_main;      /* time of the layer's main step kernel(s), timing = 1 */
    float ms_sweep;     /* converted = 3: time of the hub sweep pass alone,
                           timing = 1 or 2                                     */
    float pad;
    int64_t hub_found;  /* converted = 3: vertices found by their hub (host and
                           graph loops; 0 in the persistent device loop)       */
} bfs_layer_stats;

/* Copies up to `cap` layer records of the last run into `out`; *layers gets
 * the number of layers, *component_edges the undirected edges inside the
 * root's component (half the degree sum of the reached vertices: the TEPS
 * numerator, Sec. 6.3). Any output pointer may be NULL. */
BFS_API bfs_status bfs_last_run_stats(const bfs_graph *g, bfs_layer_stats *out, int32_t cap,
                                      int32_t *layers, int64_t *component_edges);

/* ---------------------------------------------------------------------- */
/* Batched multi-source BFS. The paper runs its 64 roots one after another */
/* (Sec. 6.3); here up to 512 roots share one traversal: root i is bit i of */
/* a per-vertex bitset, so one sweep of a vertex's row serves every root.  */
/* Each layer is the bottom-up step of Alg. 2 generalised to bit lanes (a  */
/* vertex ORs its neighbours' frontier words and stops once every lane it  */
/* still lacks is found: the paper's early exit, per lane set) or the      */
/* top-down step of Alg. 1 (frontier words ORed into neighbours' next      */
/* words), chosen per layer by the edge form of the Alg. 3 switch. A root  */
/* whose frontier empties has finished and leaves the set of live lanes.   */
/* Levels are written once, at the end, from the frontier words that every */
/* layer keeps in a ring of slots.                                         */
/* ---------------------------------------------------------------------- */
typedef struct bfs_batch_config {
    double alpha;         /* top-down -> bottom-up iff e_f > e_u / alpha, where
                             e_f = degree sum of vertices with a frontier bit
                             and e_u = degree sum of vertices still lacking
                             some live root's bit                             */
    double beta;          /* bottom-up -> top-down iff v_f < n / beta         */
    int32_t lane_probe;   /* bottom-up: neighbours a lane scans alone before
                             the warp-cooperative OR-reduction takes over     */
    int32_t big_degree;   /* top-down: largest degree threshold from which a
                             vertex's edges are spread over the grid (the
                             threshold of a layer is its frontier's edges per
                             resident row walker -- a warp for k <= 64, a
                             group of W lanes above -- clamped to
                             [32, big_degree])                               */
    int32_t use_graph;    /* 1 = run the layers as one CUDA graph with a
                             device-side loop (no per-layer host round trip) */
    int32_t timing;       /* 1 = record CUDA events per layer                 */
    int32_t layer_slots;  /* frontier slots of the level ring, 2..16 (each
                             n * W 64-bit words); 0 = as many as a quarter of
                             the free device memory holds when the bitsets are
                             allocated, 4..16. A traversal with more layers
                             than slots writes the levels of the full slots
                             before reusing them (correct, slower)           */
    int32_t reserved[7];
} bfs_batch_config;

BFS_API void bfs_batch_config_default(bfs_batch_config *cfg);
BFS_API bfs_status bfs_graph_set_batch_config(bfs_graph *g, const bfs_batch_config *cfg);
BFS_API bfs_status bfs_graph_get_batch_config(const bfs_graph *g, bfs_batch_config *cfg);

/* BFS from k roots at once (1 <= k <= 512; repeats allowed).
 *   roots        k int32 vertex ids, host or device memory
 *   levels_out   device, caller-owned, k*n int8, row i = levels from roots[i]
 *                (level[v] = hop distance, -1 when unreachable)
 * A level above 127 does not fit: the traversal stops after writing level
 * 127 and returns BFS_ERR_DEPTH (no value wraps). The bitsets (seen and the
 * frontier slots, each n * W 64-bit words with W = ceil(k/64) rounded to 1,
 * 2, 4 or 8) are allocated on first use and kept by the graph. Synchronous,
 * like bfs_run. */
BFS_API bfs_status bfs_run_batch(bfs_graph *g, const int32_t *roots, int32_t k,
                                 int8_t *levels_out, void *stream);

/* Per-layer record of the last bfs_run_batch. */
typedef struct bfs_batch_layer_stats {
    int32_t direction;   /* 0 = top-down, 1 = bottom-up                       */
    int32_t pad;
    int64_t v_f;         /* vertices holding at least one frontier bit        */
    int64_t e_f;         /* their degree sum                                  */
    int64_t pairs;       /* (root, vertex) pairs in the frontier              */
    int64_t v_u;         /* vertices of degree >= 1 still lacking some live
                            root's bit (live: its frontier is not empty)      */
    int64_t e_u;         /* their degree sum                                  */
    float ms;            /* layer time when cfg.timing = 1                    */
    float pad2;
    int64_t examined;    /* CSR entries the layer read: the rows scanned by the
                            bottom-up step up to each vertex's early exit, or
                            every frontier vertex's row in a top-down layer  */
} bfs_batch_layer_stats;

BFS_API bfs_status bfs_last_batch_stats(const bfs_graph *g, bfs_batch_layer_stats *out,
                                        int32_t cap, int32_t *layers, int64_t *pairs_reached);

/* Self-test of the grid barrier that the device-side layer loop
 * (bfs_batch_config.use_graph) synchronises with: one cooperative launch
 * waits for `missing_blocks` more blocks than it has. With 0 the barrier
 * completes (BFS_OK); with more, every block gives up after timeout_us
 * (1 ms .. 10 s) and the call returns BFS_ERR_TIMEOUT with the CUDA context
 * still usable. Failure detection on the GPU is tested this way: by a wait
 * that runs out, never by a fault. */
BFS_API bfs_status bfs_selftest_grid_barrier(int32_t missing_blocks, int64_t timeout_us,
                                             void *stream);

/* Autotuner: runs the batch from `roots` under a small grid of switch
 * thresholds (alpha, beta), lane-probe lengths and both drivers (host loop,
 * device loop), keeps the fastest in the
 * graph's batch configuration and copies it to *best (may be NULL).
 * levels_scratch is a device k*n int8 buffer it may overwrite. */
BFS_API bfs_status bfs_batch_autotune(bfs_graph *g, const int32_t *roots, int32_t k,
                                      int8_t *levels_scratch, bfs_batch_config *best,
                                      void *stream);

/* ---------------------------------------------------------------------- */
/* Serving: a request loop over resident graphs. Not in the paper (which   */
/* times one root at a time, Sec. 6.3): single-root queries are batched by  */
/* graph into bfs_run_batch launches. Worker threads, each with its own     */
/* CUDA stream, take whatever is queued whenever they are free, so queries */
/* that arrive while others run are admitted as soon as a worker and memory */
/* are free, and batches on different streams overlap on the GPU.          */
/* ---------------------------------------------------------------------- */
typedef struct bfs_server bfs_server;

typedef struct bfs_serve_config {
    int32_t workers;          /* worker threads = concurrent batches (1..16)   */
    int32_t max_batch;        /* roots per launch (1..512)                     */
    int64_t memory_budget;    /* device bytes the server may hold for batch
                                 outputs and per-worker traversal state; a
                                 batch that does not fit is halved or waits   */
    int32_t queue_capacity;   /* queued requests beyond this: BFS_ERR_BUSY     */
    int32_t cancel_on_destroy;/* 1 = queued requests end with BFS_ERR_SHUTDOWN
                                 at destroy; 0 = destroy drains them first     */
    int32_t reserved[8];
} bfs_serve_config;

typedef struct bfs_serve_stats {
    int64_t completed;        /* requests finished (any status)                */
    int64_t failed;           /* finished with a status other than BFS_OK      */
    int64_t batches;          /* bfs_run_batch launches                        */
    int64_t deferred;         /* times a batch waited for memory or was split */
    double mean_batch;        /* mean roots per launch                         */
    double p50_us, p99_us;    /* submit-to-completion latency percentiles      */
    double qps;               /* completed / (last completion - first submit)  */
    int64_t deep_fallbacks;   /* queries answered by the single-source
                                 traversal because their batch went deeper than
                                 an int8 level holds (BFS_ERR_DEPTH)           */
} bfs_serve_stats;

BFS_API void bfs_serve_config_default(bfs_serve_config *cfg);
/* Starts the workers on the current CUDA device. cfg may be NULL. */
BFS_API bfs_status bfs_serve_create(const bfs_serve_config *cfg, bfs_server **out);
/* Registers a resident graph (it must outlive the server); *graph_id names
 * it in bfs_serve_submit. Must be called before the first submit. */
BFS_API bfs_status bfs_serve_add_graph(bfs_server *s, bfs_graph *g, int32_t *graph_id);
/* Queues a BFS from `root` of graph `graph_id`. level_out: n int32, host or
 * device memory, caller-owned, written when the request completes. *ticket
 * identifies the request for bfs_serve_wait. BFS_ERR_BUSY when the queue is
 * full, BFS_ERR_SHUTDOWN after destroy began, BFS_ERR_INVALID for a bad id
 * or root. */
BFS_API bfs_status bfs_serve_submit(bfs_server *s, int32_t graph_id, int32_t root,
                                    int32_t *level_out, uint64_t *ticket);
/* Waits up to timeout_us (< 0: forever) for a ticket. Returns BFS_OK and the
 * request's own status in *result, or BFS_ERR_TIMEOUT (the ticket stays
 * valid), or BFS_ERR_INVALID for an unknown or already collected ticket. */
BFS_API bfs_status bfs_serve_wait(bfs_server *s, uint64_t ticket, int64_t timeout_us,
                                  bfs_status *result);
BFS_API bfs_status bfs_serve_stats_get(bfs_server *s, bfs_serve_stats *out);
/* Starts the statistics afresh (counts, latencies, the queries/s window);
 * requests in flight are counted when they complete. Graph views and their
 * traversal state stay allocated, so a long-running server can report one
 * interval at a time without paying their creation again. */
BFS_API bfs_status bfs_serve_stats_reset(bfs_server *s);
/* Stops accepting requests, drains or cancels the queue (cfg), finishes the
 * batches in flight, joins the workers and frees the server. NULL is fine. */
BFS_API bfs_status bfs_serve_destroy(bfs_server *s);

/* ---------------------------------------------------------------------- */
/* Allocation-free traversal. The paper has no counterpart: this entry     */
/* point exists for callers that must not allocate device memory.         */
/* ---------------------------------------------------------------------- */
/* Some callers cannot call cudaMalloc: a plugin handed only a stream by its
 * host process, a service whose device memory is owned by another allocator
 * (a framework's caching pool that has reserved the GPU), or code on a
 * latency-critical path where an allocation's implicit synchronisation is not
 * acceptable. bfs_run_noalloc runs the same hybrid BFS as bfs_run (default
 * configuration, edge policy, except that the bottom-up probe reads the CSR
 * only: head records would need an allocation) without creating a bfs_graph
 * and without any allocation: its bitmaps, queues and counters live in one fixed device
 * array compiled into the library (about 12.5 MiB on every GPU that loads
 * the library, held until the process exits).
 *   offsets, indices   device CSR (layout above), caller-owned, n <= 2^20
 *   nnz                must equal offsets[n] (read back and checked before
 *                      any launch: it seeds the e_u counter of the switch)
 *   level_out, parent_out   device, n int32 each, caller-owned (both needed)
 * n above 2^20, or nnz != offsets[n], gives BFS_ERR_INVALID. The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture
 * begins. Every call overwrites the part of the array it reads before
 * reading it, so nothing of a previous call leaks in; but all calls share
 * the one array, so calls whose work overlaps on the GPU (other streams,
 * other host threads) race and must be serialised by the caller.
 * Synchronous like bfs_run: it returns after the traversal, and on an error
 * it first drains `stream`, so no work of the call is left in flight. A
 * traversal whose counters never reach an empty frontier within n layers
 * returns BFS_ERR_INTERNAL.
 * Makes no cudaMalloc, cudaMallocAsync, cudaMallocHost or cudaFree call. */
BFS_API bfs_status bfs_run_noalloc(const int64_t *offsets, const int32_t *indices, int64_t n,
                                   int64_t nnz, int32_t root, int32_t *level_out,
                                   int32_t *parent_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GB300_HYBRID_BFS_H */
