/*
 * oracle.c -- the plain CPU oracle for the hybrid BFS library.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file. The GPU library never links,
 * includes or calls it, and it shares no code, header or table with the GPU
 * path: every function here is restated from the paper (Paredes, Riley,
 * Lujan, "Vectorization of Hybrid Breadth First Search on the Intel Xeon
 * Phi") or from the published definition it names, single-threaded, in the
 * order the definition states, with no blocking or fusion.
 *
 * Contents
 *   orc_sm64             SplitMix64 output stream, counter-indexed
 *                        (Steele, Lea, Flood, OOPSLA 2014).
 *   orc_relabel          seeded bijection of [0, 2^scale) used to relabel
 *                        generated vertices (Sec. 6.2: Graph500 Kronecker
 *                        graphs are randomly relabelled; our own recipe).
 *   orc_gen_edges        R-MAT / Kronecker edge list with initiator
 *                        A, B, C, D (Sec. 6.2) and the uniform
 *                        Erdos-Renyi control.
 *   orc_build_csr        symmetric CSR, self-loops dropped, rows sorted and
 *                        deduplicated (Sec. 6.2 "bidirectional",
 *                        Sec. 6.3 CSR).
 *   orc_sample_roots     distinct seeded roots of degree >= 1 (Sec. 6.3,
 *                        64 executions from random starting vertices).
 *   orc_bfs              FIFO layer-by-layer BFS: levels and parents
 *                        (Sec. 4 definition of layers and of P).
 *   orc_policy_decide    direction switch of Alg. 3 (two readings of f, g).
 *   orc_hybrid_bfs       Alg. 3 driving the top-down step of Alg. 1 and the
 *                        bottom-up step of Alg. 2, with the per-layer
 *                        counters e_f, v_f, e_u of Sec. 4.
 *   orc_check_levels     characterisation of BFS levels that holds at any
 *                        size (used where the FIFO oracle is too slow).
 *   orc_check_parents    BFS-tree invariants (Sec. 7.1: many trees are valid).
 *   orc_min_parent       smallest-id parent one level up (a deterministic tree).
 *   orc_hub              per-vertex neighbour of largest degree, the optional
 *                        first probe of the bottom-up step.
 *   orc_component_edges  undirected edges in the root's component, the TEPS
 *                        numerator (Sec. 6.3).
 *
 * Pins: every function above is checked in the CPU test suite against
 * something other than itself (published SplitMix64 outputs, closed forms,
 * brute-force all-pairs distances, the per-layer counts printed in Table 2
 * and Table 4, planted mistakes). No function is left unpinned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014): state advances by the golden gamma */
/* 0x9E3779B97F4A7C15 and each output is the "mix13" finaliser of the state.*/
/* Output i (0-based) of the stream seeded with s is therefore a pure       */
/* function of (s, i): mix(s + (i + 1) * gamma).                            */
/* ------------------------------------------------------------------------ */
uint64_t orc_sm64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Draw index at which the relabelling constants start; far above any edge
 * draw (edges use indices below m * scale < 2^40). */
#define ORC_PERM_BASE (1ull << 62)

/* Seeded bijection of [0, 2^scale): three rounds of an odd affine map
 * modulo 2^scale followed by x ^= x >> ceil(scale/2). Each round is
 * invertible on scale-bit integers, so the composition is a permutation. */
uint32_t orc_relabel(uint32_t x, int scale, uint64_t seed)
{
    uint64_t mask = (scale >= 64) ? ~0ull : ((1ull << scale) - 1u);
    int h = (scale + 1) / 2;
    uint64_t y = x;
    for (int j = 0; j < 3; ++j) {
        uint64_t a = orc_sm64(seed, ORC_PERM_BASE + 2u * (uint64_t)j) | 1u;
        uint64_t c = orc_sm64(seed, ORC_PERM_BASE + 2u * (uint64_t)j + 1u);
        y = (y * a + c) & mask;
        y ^= (y >> h);
    }
    return (uint32_t)y;
}

/* Edge generator (Sec. 6.2). kind 0 = R-MAT / Kronecker with initiator
 * probabilities A, B, C (D = 1 - A - B - C): for each of the `scale` bit
 * levels of an edge, one quadrant of the adjacency matrix is chosen with
 * those probabilities, giving one bit of the source and one of the
 * destination. The uniform draw for (edge e, level b) is the high 32 bits of
 * SplitMix64 output e*scale + b; quadrant thresholds are the integers
 * floor(p * 2^32) of the cumulative probabilities A, A+B, A+B+C. Vertices are
 * then relabelled by orc_relabel. kind 1 = Erdos-Renyi control: both
 * endpoints uniform, the top `scale` bits of outputs 2e and 2e+1.
 * Writes edges first .. first+count-1 of the m-edge list. */
void orc_gen_edges(int kind, int scale, uint64_t seed, double a, double b, double c,
                   int64_t first, int64_t count, int32_t *src, int32_t *dst)
{
    uint64_t t1 = (uint64_t)(a * 4294967296.0);
    uint64_t t2 = (uint64_t)((a + b) * 4294967296.0);
    uint64_t t3 = (uint64_t)((a + b + c) * 4294967296.0);
    for (int64_t k = 0; k < count; ++k) {
        uint64_t e = (uint64_t)(first + k);
        uint32_t s = 0, d = 0;
        if (kind == 0) {
            for (int lev = 0; lev < scale; ++lev) {
                uint64_t u = orc_sm64(seed, e * (uint64_t)scale + (uint64_t)lev) >> 32;
                uint32_t sbit, dbit;
                if (u < t1)      { sbit = 0; dbit = 0; }
                else if (u < t2) { sbit = 0; dbit = 1; }
                else if (u < t3) { sbit = 1; dbit = 0; }
                else             { sbit = 1; dbit = 1; }
                s |= sbit << lev;
                d |= dbit << lev;
            }
            s = orc_relabel(s, scale, seed);
            d = orc_relabel(d, scale, seed);
        } else {
            s = (uint32_t)(orc_sm64(seed, 2u * e) >> (64 - scale));
            d = (uint32_t)(orc_sm64(seed, 2u * e + 1u) >> (64 - scale));
        }
        src[k] = (int32_t)s;
        dst[k] = (int32_t)d;
    }
}

static int orc_cmp_u64(const void *x, const void *y)
{
    uint64_t p = *(const uint64_t *)x, q = *(const uint64_t *)y;
    return (p > q) - (p < q);
}

/* Symmetric CSR (Sec. 6.2: every generated edge is stored in both
 * directions; Sec. 6.3: Compressed Sparse Row). Self-loops are dropped, each
 * row is sorted ascending and duplicates are removed. offsets has n+1 int64
 * entries, indices room for 2m int32 entries. Returns nnz, or -1 if an
 * endpoint is outside [0, n) or memory runs out. */
int64_t orc_build_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                      int64_t *offsets, int32_t *indices)
{
    uint64_t *keys = (uint64_t *)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(uint64_t));
    if (!keys) return -1;
    int64_t k = 0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t s = src[e], d = dst[e];
        if (s < 0 || s >= n || d < 0 || d >= n) { free(keys); return -1; }
        if (s == d) continue;                       /* self-loop */
        keys[k++] = ((uint64_t)s << 32) | (uint64_t)d;   /* s -> d */
        keys[k++] = ((uint64_t)d << 32) | (uint64_t)s;   /* d -> s */
    }
    qsort(keys, (size_t)k, sizeof(uint64_t), orc_cmp_u64);
    for (int64_t v = 0; v <= n; ++v) offsets[v] = 0;
    int64_t nnz = 0;
    for (int64_t i = 0; i < k; ++i) {
        if (i > 0 && keys[i] == keys[i - 1]) continue;   /* duplicate */
        int64_t s = (int64_t)(keys[i] >> 32);
        indices[nnz++] = (int32_t)(keys[i] & 0xFFFFFFFFu);
        offsets[s + 1] += 1;                              /* degree count */
    }
    for (int64_t v = 0; v < n; ++v) offsets[v + 1] += offsets[v];
    free(keys);
    return nnz;
}

/* Roots (Sec. 6.3: 64 executions from random starting vertices; roots of
 * degree 0 would give zero TEPS, so only degree >= 1 is drawn). Candidate j
 * is SplitMix64 output j modulo n; candidates are taken in order j = 0, 1,
 * ..., skipping degree-0 vertices and repeats, until k roots are chosen or
 * max_draws candidates were seen. Returns the number of roots chosen. */
int32_t orc_sample_roots(const int64_t *offsets, int64_t n, uint64_t seed, int32_t k,
                         int64_t max_draws, int32_t *roots)
{
    int32_t got = 0;
    for (int64_t j = 0; j < max_draws && got < k; ++j) {
        int64_t r = (int64_t)(orc_sm64(seed, (uint64_t)j) % (uint64_t)n);
        if (offsets[r + 1] - offsets[r] < 1) continue;
        int dup = 0;
        for (int32_t i = 0; i < got; ++i)
            if (roots[i] == r) { dup = 1; break; }
        if (dup) continue;
        roots[got++] = (int32_t)r;
    }
    return got;
}

/* Layer-synchronous BFS as defined in Sec. 4: layer L_k is every vertex at
 * distance k from the source; the result is the predecessor list P. A FIFO
 * queue visits layers in order. level[v] = distance, -1 if unreachable;
 * parent[root] = root, parent[v] = -1 if unreachable. Returns the largest
 * level, or -1 if the root is out of range. */
int32_t orc_bfs(const int64_t *offsets, const int32_t *indices, int64_t n, int32_t root,
                int32_t *level, int32_t *parent)
{
    if (root < 0 || root >= n) return -1;
    for (int64_t v = 0; v < n; ++v) { level[v] = -1; parent[v] = -1; }
    int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!queue) return -1;
    int64_t head = 0, tail = 0;
    level[root] = 0;
    parent[root] = root;
    queue[tail++] = root;
    int32_t depth = 0;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = offsets[u]; e < offsets[u + 1]; ++e) {
            int32_t v = indices[e];
            if (level[v] == -1) {
                level[v] = level[u] + 1;
                parent[v] = u;
                if (level[v] > depth) depth = level[v];
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return depth;
}

/* Direction policies for Alg. 3. Alg. 3 compares |in| with two
 * architecture-specific functions f and g; Table 2 shows the switch back to
 * top-down happening while |in| > f, so the tests are read as hysteresis: in
 * top-down mode switch to bottom-up iff |in| > f; in bottom-up mode switch
 * back iff |in| < g.
 *   policy 0 (edge form, counters e_f and e_u of Sec. 4): f is passed as the
 *            test e_f > e_u / alpha, g as |in| < n / beta.
 *   policy 1 (vertex form read off Table 2): f = n_u >> 10 (n_u unvisited
 *            vertices), g = n >> 6, both compared with |in| = v_f.
 * Returns 1 for bottom-up, 0 for top-down. */
int32_t orc_policy_decide(int32_t policy, int32_t cur_bottom_up, int64_t n, int64_t n_f,
                          int64_t m_f, int64_t n_u, int64_t m_u, double alpha, double beta)
{
    if (policy == 1) {
        int64_t f = n_u >> 10, g = n >> 6;
        if (!cur_bottom_up) return n_f > f ? 1 : 0;
        return n_f < g ? 0 : 1;
    }
    if (!cur_bottom_up) return ((double)m_f > (double)m_u / alpha) ? 1 : 0;
    return ((double)n_f < (double)n / beta) ? 0 : 1;
}

/* Hybrid BFS of Alg. 3. Starts top-down (Alg. 3 initialises topdown=true).
 * Before each layer the policy picks the direction from the counters of the
 * frontier about to be processed: v_f = |in|, e_f = sum of degrees in `in`,
 * n_u / e_u = number / degree sum of vertices not yet visited (Sec. 4).
 *   top-down  (Alg. 1): for u in `in` (queue order), for v in Adj[u]: if v is
 *             not visited, mark it, append it to `out`, P[v] = u.
 *   bottom-up (Alg. 2): for every v not visited (ascending id), scan Adj[v]
 *             in CSR order; at the first n that is in `in`, mark v, append
 *             it to `out`, P[v] = n, stop.
 * policy 2 forces the direction of layer d to forced[d] (1 = bottom-up;
 * layers past max_levels keep the last entry).
 * hint (may be NULL): a neighbour of each vertex (-1 for none) that the
 * bottom-up step tests before the scan. A hit there ends the search with
 * P[v] = hint[v]; a miss counts one examined edge and the scan of Adj[v]
 * then runs as above, from its first entry. Levels do not depend on it
 * (Alg. 2 accepts any neighbour in `in`).
 * Per-layer outputs (layer d = the frontier of vertices at level d):
 *   dir[d] (1 = bottom-up), trace[6*d + 0..5] = n_f, m_f, n_u, m_u,
 *   edges examined while processing the layer, vertices found.
 * Edges examined: top-down counts every edge of the frontier; bottom-up counts,
 * per unvisited vertex, the edges up to and including the first frontier hit,
 * or its whole degree if none is found.
 * Returns the number of layers processed, or -1 on a bad argument or when
 * more than max_levels layers are needed. */
int32_t orc_hybrid_bfs(const int64_t *offsets, const int32_t *indices, int64_t n, int32_t root,
                       int32_t policy, double alpha, double beta, const int32_t *forced,
                       int32_t *level, int32_t *parent, int32_t *dir, int64_t *trace,
                       int32_t max_levels, const int32_t *hint)
{
    if (root < 0 || root >= n || max_levels < 1) return -1;
    char *vis = (char *)calloc((size_t)n, 1);
    char *in_set = (char *)calloc((size_t)n, 1);
    int32_t *in = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *out = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!vis || !in_set || !in || !out) {
        free(vis); free(in_set); free(in); free(out);
        return -1;
    }
    int64_t nnz = offsets[n];
    for (int64_t v = 0; v < n; ++v) { level[v] = -1; parent[v] = -1; }
    level[root] = 0;
    parent[root] = root;
    vis[root] = 1;
    int64_t n_in = 1;
    in[0] = root;
    int64_t n_f = 1, m_f = offsets[root + 1] - offsets[root];
    int64_t n_u = n - 1, m_u = nnz - m_f;
    int32_t bottom_up = 0, d = 0;
    while (n_in != 0) {
        if (d >= max_levels) { d = -1; break; }
        if (policy == 2) bottom_up = forced[d] ? 1 : 0;
        else bottom_up = orc_policy_decide(policy, bottom_up, n, n_f, m_f, n_u, m_u, alpha, beta);
        int64_t n_out = 0, examined = 0;
        if (!bottom_up) {
            for (int64_t i = 0; i < n_in; ++i) {
                int32_t u = in[i];
                for (int64_t e = offsets[u]; e < offsets[u + 1]; ++e) {
                    int32_t v = indices[e];
                    ++examined;
                    if (!vis[v]) {
                        vis[v] = 1;
                        out[n_out++] = v;
                        parent[v] = u;
                        level[v] = d + 1;
                    }
                }
            }
        } else {
            for (int64_t i = 0; i < n_in; ++i) in_set[in[i]] = 1;
            for (int64_t v = 0; v < n; ++v) {
                if (vis[v]) continue;
                if (hint && hint[v] >= 0) {
                    ++examined;
                    if (in_set[hint[v]]) {
                        vis[v] = 1;
                        out[n_out++] = (int32_t)v;
                        parent[v] = hint[v];
                        level[v] = d + 1;
                        continue;
                    }
                }
                for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
                    int32_t nb = indices[e];
                    ++examined;
                    if (in_set[nb]) {
                        vis[v] = 1;
                        out[n_out++] = (int32_t)v;
                        parent[v] = nb;
                        level[v] = d + 1;
                        break;
                    }
                }
            }
            for (int64_t i = 0; i < n_in; ++i) in_set[in[i]] = 0;
        }
        dir[d] = bottom_up;
        trace[6 * d + 0] = n_f;
        trace[6 * d + 1] = m_f;
        trace[6 * d + 2] = n_u;
        trace[6 * d + 3] = m_u;
        trace[6 * d + 4] = examined;
        trace[6 * d + 5] = n_out;
        /* getCounters for the next layer, then swap(in, out) and clear out. */
        int64_t m_new = 0;
        for (int64_t i = 0; i < n_out; ++i) m_new += offsets[out[i] + 1] - offsets[out[i]];
        n_f = n_out;
        m_f = m_new;
        n_u -= n_out;
        m_u -= m_new;
        int32_t *t = in; in = out; out = t;
        n_in = n_out;
        ++d;
    }
    free(vis); free(in_set); free(in); free(out);
    return d;
}

/* Characterisation of BFS levels that holds at any size: level is the
 * distance array of `root` iff (1) level[root] = 0; (2) for every edge (u, v)
 * both ends are unreached or both are reached with |level[u] - level[v]| <= 1;
 * (3) every reached v != root has a neighbour at level[v] - 1. (By induction
 * on d, (1)-(3) force layer d to be exactly the vertices at distance d.)
 * Returns 0 if valid, otherwise 1 + the first offending vertex. */
int64_t orc_check_levels(const int64_t *offsets, const int32_t *indices, int64_t n,
                         int32_t root, const int32_t *level)
{
    if (root < 0 || root >= n || level[root] != 0) return 1 + (int64_t)(root < 0 ? 0 : root);
    for (int64_t v = 0; v < n; ++v) {
        int32_t lv = level[v];
        if (lv < -1 || (lv == 0 && v != root)) return 1 + v;
        int has_up = 0;
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
            int32_t lu = level[indices[e]];
            if ((lv < 0) != (lu < 0)) return 1 + v;
            if (lv >= 0) {
                if (lu - lv > 1 || lv - lu > 1) return 1 + v;
                if (lu == lv - 1) has_up = 1;
            }
        }
        if (lv > 0 && !has_up) return 1 + v;
    }
    return 0;
}

static int orc_has_edge(const int64_t *offsets, const int32_t *indices, int32_t u, int32_t v)
{
    int64_t lo = offsets[u], hi = offsets[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (indices[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < offsets[u + 1] && indices[lo] == v;
}

/* BFS-tree invariants (Sec. 7.1: several trees are valid for one root):
 * parent[root] = root; for every reached v != root, p = parent[v] is in
 * range, (p, v) is an edge (binary search in the sorted row of p) and
 * level[p] = level[v] - 1; unreached v has parent -1. Returns 0 if valid,
 * otherwise 1 + the first offending vertex. */
int64_t orc_check_parents(const int64_t *offsets, const int32_t *indices, int64_t n,
                          int32_t root, const int32_t *level, const int32_t *parent)
{
    if (root < 0 || root >= n || parent[root] != root) return 1 + (int64_t)(root < 0 ? 0 : root);
    for (int64_t v = 0; v < n; ++v) {
        if (v == root) continue;
        int32_t p = parent[v];
        if (level[v] < 0) {
            if (p != -1) return 1 + v;
            continue;
        }
        if (p < 0 || p >= n) return 1 + v;
        if (level[p] != level[v] - 1) return 1 + v;
        if (!orc_has_edge(offsets, indices, p, (int32_t)v)) return 1 + v;
    }
    return 0;
}

/* Hub of each vertex: the neighbour of largest degree, the smallest id among
 * neighbours of equal degree; -1 for a vertex without neighbours. A
 * high-degree neighbour is the one most likely to be in an early frontier,
 * so it is a cheap first test for the bottom-up step (hint of
 * orc_hybrid_bfs). */
void orc_hub(const int64_t *offsets, const int32_t *indices, int64_t n, int32_t *hub)
{
    for (int64_t v = 0; v < n; ++v) {
        int32_t best = -1;
        int64_t best_deg = -1;
        for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
            int32_t u = indices[e];
            int64_t du = offsets[u + 1] - offsets[u];
            if (du > best_deg || (du == best_deg && u < best)) {
                best = u;
                best_deg = du;
            }
        }
        hub[v] = best;
    }
}

/* Smallest-id parent: for each reached v != root, the smallest neighbour u
 * with level[u] = level[v] - 1; parent[root] = root; -1 when unreached. */
void orc_min_parent(const int64_t *offsets, const int32_t *indices, int64_t n, int32_t root,
                    const int32_t *level, int32_t *parent)
{
    for (int64_t v = 0; v < n; ++v) {
        int32_t best = -1;
        if (v == root) best = root;
        else if (level[v] > 0) {
            for (int64_t e = offsets[v]; e < offsets[v + 1]; ++e) {
                int32_t u = indices[e];
                if (level[u] == level[v] - 1 && (best < 0 || u < best)) best = u;
            }
        }
        parent[v] = best;
    }
}

/* TEPS numerator (Sec. 6.3): undirected, deduplicated edges inside the
 * root's component, i.e. half the degree sum over reached vertices. */
int64_t orc_component_edges(const int64_t *offsets, int64_t n, const int32_t *level)
{
    int64_t s = 0;
    for (int64_t v = 0; v < n; ++v)
        if (level[v] >= 0) s += offsets[v + 1] - offsets[v];
    return s / 2;
}
