// Continuous-batching BFS server over several resident graphs.
//
// Queries (graph, source, output row) queue per graph.  A fixed set of slots --
// each a CUDA stream with its own workspace (the persistent kernels' scratch),
// staging buffers and completion event -- runs batches: whenever a slot is free,
// the graph whose oldest query has waited longest sends up to its lane width of
// queued queries as one batched BFS (gbx_bfs_batch's kernel), every lane writing
// straight into its query's output row.  Each slot's persistent kernel gets
// 1/slots of the GPU's resident blocks, so batches -- of different graphs or of
// the same graph -- run side by side.  Queries that arrive while batches are in
// flight join the next batch as soon as a slot frees up.  Admission: a graph's
// lane width is capped so that the slots' batch scratch stays within the memory
// budget, and submissions beyond max_pending queued queries are refused with
// GBX_ERR_BUSY.
#include <chrono>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include "gbx_internal.cuh"

namespace gbx {

struct Query {
    int32_t graph;
    int32_t source;
    void* out;
    uint64_t tag;
    double t_submit;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int32_t* src_dev = nullptr;
    void** rows_dev = nullptr;
    int32_t* src_pinned = nullptr;
    void** rows_pinned = nullptr;
    int32_t* status_pinned = nullptr;
    Workspace ws;
    std::vector<Query> batch;
    int graph = -1;
    bool busy = false;
    double t_launch = 0.0;
};

struct GraphEntry {
    Graph* g = nullptr;
    int32_t lanes = 0;
    gbx_desc desc;  // descriptor of this graph's batches (direction threshold, lane probe)
    std::deque<Query> pending;
};

struct Server {
    gbx_server_config cfg;
    std::vector<GraphEntry> graphs;
    std::vector<Slot> slots;
    int64_t scratch_bytes = 0;  // batch scratch of one slot (all slots hold the same)
    int64_t queued = 0;
    int64_t rejected = 0;
    std::chrono::steady_clock::time_point t0;
    std::deque<gbx_completion> done;
    std::mutex mu;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

static void server_release(Server* S) {
    if (!S) return;
    for (Slot& sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.src_dev) cudaFree(sl.src_dev);
        if (sl.rows_dev) cudaFree(sl.rows_dev);
        if (sl.src_pinned) cudaFreeHost(sl.src_pinned);
        if (sl.rows_pinned) cudaFreeHost(sl.rows_pinned);
        if (sl.status_pinned) cudaFreeHost(sl.status_pinned);
        workspace_release(sl.ws);
    }
    delete S;
}

// Completed batches -> completion records; the slot becomes free again.
static gbx_status reap(Server* S) {
    for (Slot& sl : S->slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        GBX_CUDA_TRY(q);
        const double t = S->now();
        const int32_t err = sl.status_pinned[ST_ERROR];
        if (err != 0) {  // clear the recorded error and the barrier the kernel may have left
            GBX_CUDA_TRY(cudaMemsetAsync(sl.ws.status + ST_ERROR, 0, sizeof(int32_t), sl.stream));
            GBX_CUDA_TRY(cudaMemsetAsync(sl.ws.bar, 0, sizeof(GridBar), sl.stream));
            GBX_CUDA_TRY(cudaStreamSynchronize(sl.stream));
        }
        for (const Query& qq : sl.batch) {
            gbx_completion c = {};
            c.tag = qq.tag;
            c.graph_id = qq.graph;
            c.source = qq.source;
            c.status = err;
            c.levels = sl.status_pinned[ST_LEVELS];
            c.batch_size = (int32_t)sl.batch.size();
            c.t_submit = qq.t_submit;
            c.t_launch = sl.t_launch;
            c.t_done = t;
            S->done.push_back(c);
        }
        sl.batch.clear();
        sl.busy = false;
    }
    return GBX_OK;
}

// Copies a slot's staged sources and output rows, launches its batch and queues the
// status read-back and the completion event, all on the slot's stream.
static gbx_status launch_batch(Server* S, Slot& sl, const GraphEntry& ge, int32_t nb) {
    GBX_CUDA_TRY(cudaMemcpyAsync(sl.src_dev, sl.src_pinned, sizeof(int32_t) * nb, cudaMemcpyHostToDevice, sl.stream));
    GBX_CUDA_TRY(cudaMemcpyAsync(sl.rows_dev, sl.rows_pinned, sizeof(void*) * nb, cudaMemcpyHostToDevice, sl.stream));
    GBX_TRY(ms_run(ge.g, sl.ws, nb, sl.src_dev, nullptr, sl.rows_dev, S->cfg.depth_type == GBX_DEPTH_I16 ? 1 : 0,
                   ge.desc, (int)S->slots.size(), sl.stream));
    GBX_CUDA_TRY(cudaMemcpyAsync(sl.status_pinned, sl.ws.status, sizeof(int32_t) * ST_WORDS, cudaMemcpyDeviceToHost,
                                 sl.stream));
    GBX_CUDA_TRY(cudaEventRecord(sl.done, sl.stream));
    return GBX_OK;
}

// Start batches on free slots, oldest waiting graph first.  A batch whose launch
// fails completes at once: each of its queries gets a completion carrying the error
// (and gbx_last_error its message), so no accepted query is ever dropped.
static gbx_status dispatch(Server* S) {
    for (Slot& sl : S->slots) {
        if (sl.busy) continue;
        int best = -1;
        double best_t = 0.0;
        for (int i = 0; i < (int)S->graphs.size(); ++i) {
            const GraphEntry& ge = S->graphs[i];
            if (ge.pending.empty()) continue;
            if (best < 0 || ge.pending.front().t_submit < best_t) {
                best = i;
                best_t = ge.pending.front().t_submit;
            }
        }
        if (best < 0) return GBX_OK;
        GraphEntry& ge = S->graphs[best];
        const int32_t nb = (int32_t)(ge.pending.size() < (size_t)ge.lanes ? ge.pending.size() : (size_t)ge.lanes);
        sl.batch.clear();
        for (int32_t k = 0; k < nb; ++k) {
            const Query qq = ge.pending.front();
            ge.pending.pop_front();
            sl.src_pinned[k] = qq.source;
            sl.rows_pinned[k] = qq.out;
            sl.batch.push_back(qq);
        }
        S->queued -= nb;
        sl.t_launch = S->now();
        const gbx_status st = launch_batch(S, sl, ge, nb);
        if (st != GBX_OK) {
            const double t = S->now();
            for (const Query& qq : sl.batch) {
                gbx_completion c = {};
                c.tag = qq.tag;
                c.graph_id = qq.graph;
                c.source = qq.source;
                c.status = st;
                c.levels = 0;
                c.batch_size = nb;
                c.t_submit = qq.t_submit;
                c.t_launch = sl.t_launch;
                c.t_done = t;
                S->done.push_back(c);
            }
            sl.batch.clear();
            continue;
        }
        sl.graph = best;
        sl.busy = true;
    }
    return GBX_OK;
}

}  // namespace gbx

using namespace gbx;

extern "C" void gbx_server_config_init(gbx_server_config* c) {
    if (!c) return;
    *c = gbx_server_config{};
    c->max_batch = 64;
    c->max_pending = 1 << 16;
    c->memory_budget = 0;
    c->slots = 2;
    c->depth_type = GBX_DEPTH_I32;
    c->alpha = 0.05f;
}

extern "C" gbx_status gbx_server_create(gbx_server** out, const gbx_server_config* cfg) {
    clear_error();
    GBX_CHECK(out != nullptr, GBX_ERR_NULL_POINTER, "out is NULL");
    *out = nullptr;
    gbx_server_config c;
    if (cfg)
        c = *cfg;
    else
        gbx_server_config_init(&c);
    GBX_CHECK(c.max_batch >= 1 && c.max_batch <= 4096, GBX_ERR_INVALID_VALUE, "max_batch must be in [1, 4096]");
    GBX_CHECK(c.slots >= 1 && c.slots <= 16, GBX_ERR_INVALID_VALUE, "slots must be in [1, 16]");
    GBX_CHECK(c.max_pending >= 1, GBX_ERR_INVALID_VALUE, "max_pending must be >= 1");
    GBX_CHECK(c.memory_budget >= 0, GBX_ERR_INVALID_VALUE, "memory_budget must be >= 0");
    GBX_CHECK(c.depth_type == GBX_DEPTH_I32 || c.depth_type == GBX_DEPTH_I16, GBX_ERR_INVALID_VALUE, "depth_type");
    GBX_CHECK(c.alpha >= 0.0f && c.alpha == c.alpha, GBX_ERR_INVALID_VALUE, "alpha must be >= 0");
    for (int k = 0; k < 4; ++k) GBX_CHECK(c.reserved[k] == 0, GBX_ERR_INVALID_VALUE, "reserved must be 0");
    Server* S = new (std::nothrow) Server();
    GBX_CHECK(S != nullptr, GBX_ERR_OUT_OF_MEMORY, "host allocation failed");
    S->cfg = c;
    S->t0 = std::chrono::steady_clock::now();
    S->slots.resize(c.slots);
    for (Slot& sl : S->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc((void**)&sl.src_dev, sizeof(int32_t) * c.max_batch);
        if (e == cudaSuccess) e = cudaMalloc((void**)&sl.rows_dev, sizeof(void*) * c.max_batch);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.src_pinned, sizeof(int32_t) * c.max_batch);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.rows_pinned, sizeof(void*) * c.max_batch);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.status_pinned, sizeof(int32_t) * ST_WORDS);
        if (e != cudaSuccess) {
            server_release(S);
            GBX_CUDA_TRY(e);
        }
    }
    *out = reinterpret_cast<gbx_server*>(S);
    return GBX_OK;
}

extern "C" gbx_status gbx_server_add_graph(gbx_server* srv, gbx_graph* g, int32_t* graph_id) {
    clear_error();
    GBX_CHECK(srv != nullptr && g != nullptr && graph_id != nullptr, GBX_ERR_NULL_POINTER, "NULL argument");
    Server* S = reinterpret_cast<Server*>(srv);
    std::lock_guard<std::mutex> lock(S->mu);
    Graph* G = as_impl(g);
    for (const GraphEntry& ge : S->graphs) GBX_CHECK(ge.g != G, GBX_ERR_INVALID_VALUE, "graph already added");
    const int64_t nslots = (int64_t)S->slots.size();
    // lane width: the largest multiple of 64 (or max_batch) whose scratch, held once
    // per slot, fits the budget together with what the other graphs need
    int32_t lanes = S->cfg.max_batch;
    if (S->cfg.memory_budget > 0) {
        auto need = [&](int32_t l) {
            const int64_t b = ms_scratch_bytes(G->n, l);
            return nslots * (b > S->scratch_bytes ? b : S->scratch_bytes);
        };
        while (lanes > 0 && need(lanes) > S->cfg.memory_budget) lanes = lanes > 64 ? (lanes - 1) / 64 * 64 : lanes - 1;
        GBX_CHECK(lanes >= 1, GBX_ERR_OUT_OF_MEMORY, "memory budget too small for this graph");
    }
    for (Slot& sl : S->slots) {
        if (sl.ws.n_cap < G->n) {  // grow the slot's workspace to this graph's size
            GBX_CUDA_TRY(cudaStreamSynchronize(sl.stream));
            const int64_t cap = sl.ws.ms_cap_words;
            workspace_release(sl.ws);
            GBX_TRY(workspace_alloc(sl.ws, G->n));
            (void)cap;
        }
        GBX_TRY(ms_reserve(sl.ws, G->n, lanes, sl.stream));
    }
    for (const GraphEntry& ge : S->graphs)
        for (Slot& sl : S->slots) GBX_TRY(ms_reserve(sl.ws, ge.g->n, ge.lanes, sl.stream));
    const int64_t b = ms_scratch_bytes(G->n, lanes);
    if (b > S->scratch_bytes) S->scratch_bytes = b;
    GraphEntry ge;
    ge.g = G;
    ge.lanes = lanes;
    gbx_desc_init(&ge.desc);
    ge.desc.alpha = S->cfg.alpha;
    S->graphs.push_back(ge);
    *graph_id = (int32_t)S->graphs.size() - 1;
    return GBX_OK;
}

extern "C" gbx_status gbx_server_graph_lanes(gbx_server* srv, int32_t graph_id, int32_t* lanes) {
    clear_error();
    GBX_CHECK(srv != nullptr && lanes != nullptr, GBX_ERR_NULL_POINTER, "NULL argument");
    Server* S = reinterpret_cast<Server*>(srv);
    std::lock_guard<std::mutex> lock(S->mu);
    GBX_CHECK(graph_id >= 0 && graph_id < (int32_t)S->graphs.size(), GBX_ERR_INVALID_INDEX, "unknown graph id");
    *lanes = S->graphs[graph_id].lanes;
    return GBX_OK;
}

extern "C" gbx_status gbx_server_set_graph_desc(gbx_server* srv, int32_t graph_id, const gbx_desc* desc) {
    clear_error();
    GBX_CHECK(srv != nullptr && desc != nullptr, GBX_ERR_NULL_POINTER, "NULL argument");
    Server* S = reinterpret_cast<Server*>(srv);
    std::lock_guard<std::mutex> lock(S->mu);
    GBX_CHECK(graph_id >= 0 && graph_id < (int32_t)S->graphs.size(), GBX_ERR_INVALID_INDEX, "unknown graph id");
    const gbx_desc& d = *desc;
    GBX_CHECK(d.direction >= GBX_DIR_AUTO && d.direction <= GBX_DIR_PULL, GBX_ERR_INVALID_VALUE, "desc.direction");
    GBX_CHECK(d.alpha >= 0.0f && d.alpha == d.alpha, GBX_ERR_INVALID_VALUE, "desc.alpha must be >= 0");
    GBX_CHECK(d.pull_probe == 0 || (d.pull_probe >= 4 && d.pull_probe <= 1024), GBX_ERR_INVALID_VALUE,
              "desc.pull_probe must be 0 or in [4, 1024]");
    GBX_CHECK(d.push_sort == 0, GBX_ERR_NOT_SUPPORTED, "desc.push_sort applies to gbx_mxv only");
    GBX_CHECK(d.blocks_per_sm >= 0, GBX_ERR_INVALID_VALUE, "desc.blocks_per_sm must be >= 0");
    gbx_desc keep = d;
    keep.trace = 0;  // batches of the server are not traced
    S->graphs[graph_id].desc = keep;
    return GBX_OK;
}

extern "C" gbx_status gbx_server_submit(gbx_server* srv, int32_t graph_id, int32_t source, void* depth_out,
                                        uint64_t tag) {
    clear_error();
    GBX_CHECK(srv != nullptr && depth_out != nullptr, GBX_ERR_NULL_POINTER, "NULL argument");
    Server* S = reinterpret_cast<Server*>(srv);
    std::lock_guard<std::mutex> lock(S->mu);
    GBX_CHECK(graph_id >= 0 && graph_id < (int32_t)S->graphs.size(), GBX_ERR_INVALID_INDEX, "unknown graph id");
    GraphEntry& ge = S->graphs[graph_id];
    GBX_CHECK(source >= 0 && source < ge.g->n, GBX_ERR_INVALID_INDEX, "source outside [0, n)");
    if (S->queued >= S->cfg.max_pending) {
        S->rejected += 1;
        set_error("server queue full");
        return GBX_ERR_BUSY;
    }
    ge.pending.push_back(Query{graph_id, source, depth_out, tag, S->now()});
    S->queued += 1;
    GBX_TRY(reap(S));
    return dispatch(S);
}

extern "C" gbx_status gbx_server_poll(gbx_server* srv, gbx_completion* out, int32_t max, int32_t* nout) {
    clear_error();
    GBX_CHECK(srv != nullptr && nout != nullptr, GBX_ERR_NULL_POINTER, "NULL argument");
    GBX_CHECK(max == 0 || out != nullptr, GBX_ERR_NULL_POINTER, "out is NULL");
    Server* S = reinterpret_cast<Server*>(srv);
    std::lock_guard<std::mutex> lock(S->mu);
    GBX_TRY(reap(S));
    GBX_TRY(dispatch(S));
    int32_t k = 0;
    while (k < max && !S->done.empty()) {
        out[k++] = S->done.front();
        S->done.pop_front();
    }
    *nout = k;
    return GBX_OK;
}

extern "C" gbx_status gbx_server_stats(gbx_server* srv, int64_t* queued, int32_t* in_flight, int64_t* rejected,
                                       int64_t* scratch_bytes) {
    clear_error();
    GBX_CHECK(srv != nullptr, GBX_ERR_NULL_POINTER, "NULL argument");
    Server* S = reinterpret_cast<Server*>(srv);
    std::lock_guard<std::mutex> lock(S->mu);
    int32_t busy = 0;
    for (const Slot& sl : S->slots) busy += sl.busy ? (int32_t)sl.batch.size() : 0;
    if (queued) *queued = S->queued;
    if (in_flight) *in_flight = busy;
    if (rejected) *rejected = S->rejected;
    if (scratch_bytes) *scratch_bytes = S->scratch_bytes * (int64_t)S->slots.size();
    return GBX_OK;
}

extern "C" gbx_status gbx_server_destroy(gbx_server* srv) {
    clear_error();
    if (!srv) return GBX_OK;
    server_release(reinterpret_cast<Server*>(srv));
    return GBX_OK;
}
