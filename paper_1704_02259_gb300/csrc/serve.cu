// serve.cu -- request loop over resident graphs with continuous batching.
//
// Requests (graph, root, output) wait in one FIFO per graph. Each worker
// thread owns a CUDA stream and, per graph, a view of the registered graph
// (same CSR, borrowed, with its own traversal state). A free worker picks
// the graph whose oldest request waited longest, takes up to max_batch of
// its requests, reserves device memory for the batch against the server's
// budget (halving the batch, or waiting for other batches to release memory,
// when it does not fit), runs one bfs_run_batch, expands each root's int8
// row into the requester's int32 levels, and completes the tickets. Requests
// arriving meanwhile are taken by whichever worker frees up next, so batches
// on different streams overlap on the GPU.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace gbfs {
namespace {

using clk = std::chrono::steady_clock;

struct Req {
    uint64_t ticket = 0;
    int32_t graph = 0;
    int32_t root = 0;
    int32_t *out = nullptr;
    bool out_host = false;
    clk::time_point t_submit;
    bfs_status status = BFS_OK;
    bool done = false;
};

struct GraphEntry {
    bfs_graph *g = nullptr;
    const int64_t *off = nullptr;
    const int32_t *idx = nullptr;
    int64_t n = 0, nnz = 0;
    std::deque<Req *> q;
};

__global__ void unpack_row_kernel(const int8_t *__restrict__ row, int64_t n,
                                  int32_t *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = row[i];
}

// Device bytes a worker's view of an n-vertex graph holds: the single-source
// scratch (bitmaps, queues, the parent scratch of the depth fallback) plus the
// batched lists; view_lane_bytes adds the bitsets for W lane words.
int64_t view_base_bytes(int64_t n) { return 26 * n + (1 << 16); }
// seen and kViewSlots frontier slots of n * W 64-bit words
constexpr int kViewSlots = 8;
int64_t view_lane_bytes(int64_t n, int W) { return 8 * (1 + kViewSlots) * n * (int64_t)W; }
int lane_words(int k) { return k <= 64 ? 1 : k <= 128 ? 2 : k <= 256 ? 4 : 8; }

bool host_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

}  // namespace
}  // namespace gbfs

using namespace gbfs;

struct bfs_server {
    bfs_serve_config cfg;
    int device = 0;
    std::vector<GraphEntry> graphs;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_mem;
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_ticket = 1;
    bool stopping = false;
    int64_t queued = 0;
    int64_t mem_used = 0;
    int running = 0;
    std::vector<std::thread> workers;
    std::vector<double> lat_us;
    int64_t completed = 0, failed = 0, batches = 0, deferred = 0, roots_launched = 0;
    int64_t deep_fallbacks = 0;
    bool any_submit = false;
    clk::time_point first_submit, last_done;
};

namespace gbfs {
namespace {

void finish(bfs_server *s, Req *r, bfs_status st, clk::time_point now) {
    r->status = st;
    r->done = true;
    s->completed += 1;
    if (st != BFS_OK) s->failed += 1;
    s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r->t_submit).count());
    s->last_done = now;
}

void worker_main(bfs_server *s, int wid) {
    (void)wid;
    cudaSetDevice(s->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    std::vector<bfs_graph *> views;
    std::vector<int> view_w;
    int32_t *staging = nullptr;
    int64_t staging_n = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_work.wait(lk, [&] { return s->queued > 0 || s->stopping; });
        if (s->queued == 0) {
            if (s->stopping) break;
            continue;
        }
        // the graph whose oldest request has waited longest
        int gi = -1;
        for (int i = 0; i < (int)s->graphs.size(); ++i)
            if (!s->graphs[i].q.empty() &&
                (gi < 0 || s->graphs[i].q.front()->t_submit < s->graphs[gi].q.front()->t_submit))
                gi = i;
        if (gi < 0) continue;
        GraphEntry &ge = s->graphs[gi];
        if ((int)views.size() <= gi) {
            views.resize(gi + 1, nullptr);
            view_w.resize(gi + 1, 0);
        }
        int k = (int)std::min<int64_t>(s->cfg.max_batch, (int64_t)ge.q.size());
        auto need_of = [&](int kk) {
            int64_t b = (int64_t)kk * ge.n;  // int8 level rows
            if (!views[gi]) b += view_base_bytes(ge.n);
            const int w = lane_words(kk);
            if (w > view_w[gi]) b += view_lane_bytes(ge.n, w) - view_lane_bytes(ge.n, view_w[gi]);
            if (staging_n < ge.n) b += 4 * (ge.n - staging_n);
            return b;
        };
        int64_t need = need_of(k);
        bool admitted = true;
        while (s->mem_used + need > s->cfg.memory_budget) {
            if (k > 1) {
                k = (k + 1) / 2;
                need = need_of(k);
                s->deferred += 1;
                continue;
            }
            if (s->running == 0) {  // nothing in flight will free memory
                Req *r = ge.q.front();
                ge.q.pop_front();
                s->queued -= 1;
                finish(s, r, BFS_ERR_OOM, clk::now());
                s->cv_done.notify_all();
                admitted = false;
                break;
            }
            s->deferred += 1;
            s->cv_mem.wait(lk);
            admitted = false;  // re-pick: the queues may have changed
            break;
        }
        if (!admitted) continue;
        std::vector<Req *> batch(ge.q.begin(), ge.q.begin() + k);
        ge.q.erase(ge.q.begin(), ge.q.begin() + k);
        s->queued -= k;
        s->mem_used += need;
        s->running += 1;
        s->batches += 1;
        s->roots_launched += k;
        const int64_t n = ge.n, nnz = ge.nnz;
        const int64_t *g_off = ge.off;
        const int32_t *g_idx = ge.idx;
        bfs_graph *const g_src = ge.g;
        const int64_t rows_bytes = (int64_t)k * n;
        const int64_t keep_bytes = need - rows_bytes;
        lk.unlock();

        bfs_status status = BFS_OK;
        if (!views[gi]) {
            bfs_graph *v = nullptr;
            bfs_config vc;  // a view runs batches only: no single-source head records
            bfs_config_default(&vc);
            vc.bu_head = 0;
            status = bfs_graph_create(g_off, g_idx, n, nnz, BFS_DEVICE_PTRS | BFS_BORROW, &vc,
                                      &v);
            // the single-source fallback below then allocates nothing
            if (status == BFS_OK) status = bfs_graph_reserve(v, BFS_RESERVE_NO_PARENT, st);
            if (status != BFS_OK && v) {
                bfs_graph_destroy(v);
                v = nullptr;
            }
            if (status == BFS_OK) {
                bfs_batch_config bc;
                bfs_graph_get_batch_config(g_src, &bc);
                bc.timing = 0;
                bc.layer_slots = kViewSlots;
                bfs_graph_set_batch_config(v, &bc);
                views[gi] = v;
            }
        }
        if (status == BFS_OK && staging_n < n) {
            cudaFree(staging);
            staging = nullptr;
            staging_n = 0;
            if (dev_malloc(&staging, (size_t)n * 4) == cudaSuccess) staging_n = n;
            else status = BFS_ERR_OOM;
        }
        int8_t *rows = nullptr;
        if (status == BFS_OK && dev_malloc_async(&rows, (size_t)rows_bytes, st) != cudaSuccess) {
            cudaGetLastError();
            status = BFS_ERR_OOM;
        }
        if (status == BFS_OK) {
            std::vector<int32_t> roots(k);
            for (int i = 0; i < k; ++i) roots[i] = batch[i]->root;
            status = bfs_run_batch(views[gi], roots.data(), k, rows, st);
            if (status == BFS_OK) view_w[gi] = std::max(view_w[gi], lane_words(k));
        }
        int deep = 0;
        if (status == BFS_ERR_DEPTH) {
            // The batch went deeper than an int8 level holds (127): each of
            // its queries is answered by the single-source traversal, which
            // has no depth limit and writes int32 levels directly.
            status = BFS_OK;
            for (int i = 0; i < k && status == BFS_OK; ++i) {
                Req *r = batch[i];
                int32_t *dst = r->out_host ? staging : r->out;
                status = bfs_run(views[gi], r->root, dst, nullptr, st);
                if (status == BFS_OK && r->out_host &&
                    cudaMemcpyAsync(r->out, staging, (size_t)n * 4, cudaMemcpyDeviceToHost, st) !=
                        cudaSuccess)
                    status = BFS_ERR_CUDA;
            }
            deep = k;
        } else if (status == BFS_OK) {
            const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
            for (int i = 0; i < k && status == BFS_OK; ++i) {
                Req *r = batch[i];
                int32_t *dst = r->out_host ? staging : r->out;
                unpack_row_kernel<<<grid, 256, 0, st>>>(rows + (int64_t)i * n, n, dst);
                count_launch();
                if (cudaGetLastError() != cudaSuccess) status = BFS_ERR_CUDA;
                if (r->out_host &&
                    cudaMemcpyAsync(r->out, staging, (size_t)n * 4, cudaMemcpyDeviceToHost, st) !=
                        cudaSuccess)
                    status = BFS_ERR_CUDA;
            }
        }
        if (rows) cudaFreeAsync(rows, st);
        if (cudaStreamSynchronize(st) != cudaSuccess && status == BFS_OK) status = BFS_ERR_CUDA;

        lk.lock();
        s->mem_used -= rows_bytes;
        if (status != BFS_OK) s->mem_used -= keep_bytes;  // nothing new is kept on failure
        s->running -= 1;
        s->deep_fallbacks += deep;
        const clk::time_point now = clk::now();
        for (Req *r : batch) finish(s, r, status, now);
        s->cv_done.notify_all();
        s->cv_mem.notify_all();
    }
    lk.unlock();
    for (bfs_graph *v : views) bfs_graph_destroy(v);
    cudaFree(staging);
    cudaStreamDestroy(st);
}

}  // namespace
}  // namespace gbfs

extern "C" BFS_API void bfs_serve_config_default(bfs_serve_config *c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->workers = 4;
    c->max_batch = 512;
    c->memory_budget = 64ll << 30;
    c->queue_capacity = 1 << 20;
    c->cancel_on_destroy = 0;
}

extern "C" BFS_API bfs_status bfs_serve_create(const bfs_serve_config *cfg, bfs_server **out) {
    clear_error();
    if (!out) {
        set_error("bfs_serve_create: null output");
        return BFS_ERR_INVALID;
    }
    bfs_serve_config c;
    if (cfg) c = *cfg;
    else bfs_serve_config_default(&c);
    if (c.workers < 1 || c.workers > 16 || c.max_batch < 1 || c.max_batch > 512 ||
        c.memory_budget < 0 || c.queue_capacity < 1) {
        set_error("bfs_serve_create: invalid configuration");
        return BFS_ERR_INVALID;
    }
    bfs_server *s = new bfs_server();
    s->cfg = c;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        set_error("bfs_serve_create: no CUDA device");
        return BFS_ERR_CUDA;
    }
    for (int i = 0; i < c.workers; ++i) s->workers.emplace_back(worker_main, s, i);
    *out = s;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_serve_add_graph(bfs_server *s, bfs_graph *g, int32_t *graph_id) {
    clear_error();
    if (!s || !g || !graph_id) {
        set_error("bfs_serve_add_graph: null argument");
        return BFS_ERR_INVALID;
    }
    GraphEntry e;
    e.g = g;
    bfs_status st = bfs_graph_info(g, &e.off, &e.idx, &e.n, &e.nnz);
    if (st != BFS_OK) return st;
    std::lock_guard<std::mutex> lk(s->mu);
    s->graphs.push_back(std::move(e));
    *graph_id = (int32_t)s->graphs.size() - 1;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_serve_submit(bfs_server *s, int32_t graph_id, int32_t root,
                                               int32_t *level_out, uint64_t *ticket) {
    clear_error();
    if (!s || !level_out || !ticket) {
        set_error("bfs_serve_submit: null argument");
        return BFS_ERR_INVALID;
    }
    const bool out_host = host_ptr(level_out);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) {
        set_error("bfs_serve_submit: the server is shutting down");
        return BFS_ERR_SHUTDOWN;
    }
    if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size() || root < 0 ||
        root >= s->graphs[graph_id].n) {
        set_error("bfs_serve_submit: unknown graph id or root out of range");
        return BFS_ERR_INVALID;
    }
    if (s->queued >= s->cfg.queue_capacity) {
        set_error("bfs_serve_submit: queue full");
        return BFS_ERR_BUSY;
    }
    Req *r = new Req();
    r->ticket = s->next_ticket++;
    r->graph = graph_id;
    r->root = root;
    r->out = level_out;
    r->out_host = out_host;
    r->t_submit = clk::now();
    if (!s->any_submit) {
        s->any_submit = true;
        s->first_submit = r->t_submit;
    }
    s->reqs[r->ticket] = r;
    s->graphs[graph_id].q.push_back(r);
    s->queued += 1;
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_serve_wait(bfs_server *s, uint64_t ticket, int64_t timeout_us,
                                             bfs_status *result) {
    clear_error();
    if (!s) {
        set_error("bfs_serve_wait: null server");
        return BFS_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("bfs_serve_wait: unknown or already collected ticket");
        return BFS_ERR_INVALID;
    }
    Req *r = it->second;
    if (timeout_us < 0) {
        s->cv_done.wait(lk, [&] { return r->done; });
    } else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us),
                                    [&] { return r->done; })) {
        set_error("bfs_serve_wait: timed out");
        return BFS_ERR_TIMEOUT;
    }
    if (result) *result = r->status;
    s->reqs.erase(ticket);
    delete r;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_serve_stats_get(bfs_server *s, bfs_serve_stats *o) {
    clear_error();
    if (!s || !o) {
        set_error("bfs_serve_stats_get: null argument");
        return BFS_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    memset(o, 0, sizeof *o);
    o->completed = s->completed;
    o->failed = s->failed;
    o->batches = s->batches;
    o->deferred = s->deferred;
    o->deep_fallbacks = s->deep_fallbacks;
    o->mean_batch = s->batches ? (double)s->roots_launched / s->batches : 0.0;
    if (!s->lat_us.empty()) {
        std::vector<double> v = s->lat_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            size_t i = (size_t)std::min<double>(v.size() - 1, std::max(0.0, p * v.size() - 1e-9));
            return v[i];
        };
        o->p50_us = pct(0.50);
        o->p99_us = pct(0.99);
        const double span = std::chrono::duration<double>(s->last_done - s->first_submit).count();
        o->qps = span > 0 ? s->completed / span : 0.0;
    }
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_serve_stats_reset(bfs_server *s) {
    clear_error();
    if (!s) {
        set_error("bfs_serve_stats_reset: null server");
        return BFS_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_us.clear();
    s->completed = s->failed = s->batches = s->deferred = s->roots_launched = 0;
    s->deep_fallbacks = 0;
    s->any_submit = false;
    return BFS_OK;
}

extern "C" BFS_API bfs_status bfs_serve_destroy(bfs_server *s) {
    clear_error();
    if (!s) return BFS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        if (s->cfg.cancel_on_destroy) {
            const clk::time_point now = clk::now();
            for (GraphEntry &ge : s->graphs) {
                for (Req *r : ge.q) finish(s, r, BFS_ERR_SHUTDOWN, now);
                ge.q.clear();
            }
            s->queued = 0;
            s->cv_done.notify_all();
        }
    }
    s->cv_work.notify_all();
    s->cv_mem.notify_all();
    for (std::thread &t : s->workers) t.join();
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return BFS_OK;
}
