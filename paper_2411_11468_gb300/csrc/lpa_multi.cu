// Batches of independent graphs and the request server: several resident graphs share one
// launch plan, so each sweep kernel covers the vertices of every graph while each graph keeps
// its own run state (sweep index, Pick-Less phase, changed count, stop decision).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lpa_graph_internal.h"

using namespace lpa;

namespace {

// Fresh run of every graph of a plan (blockIdx.y: graph): labels = vertex ids, every vertex
// with an edge unprocessed, counters and mover counts zeroed.
__global__ void k_init_multi(const GraphDev *gd)
{
    const GraphDev &G = gd[blockIdx.y];
    const RunState *rs = G.rs;
    if (rs->done) return;
    const int64_t n = rs->n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        G.C[i] = (int32_t)i;
        G.flags0[i] = G.off[i + 1] > G.off[i] ? 1 : 0;
        G.flags1[i] = 0;
    }
    const int64_t words = (int64_t)G.ctr_iters * kPerSweep;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < words; q += (int64_t)gridDim.x * blockDim.x)
        G.ctr[q] = 0ull;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        G.mover_count[0] = 0ull;
        G.mover_count[1] = 0ull;
        *G.fallbacks = 0ull;
    }
}

template <typename T>
int grow(T **p, size_t *cap, size_t need)
{
    if (need <= *cap && *p) return LPA_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    const size_t c = std::max<size_t>(need, 16) * 3 / 2;
    if (cudaMalloc((void **)p, c * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("cudaMalloc for a launch plan failed");
        return LPA_ENOMEM;
    }
    *cap = c;
    return LPA_OK;
}

// The combined launch plan of a set of resident graphs.
struct MultiPlan {
    cudaStream_t stream = nullptr;
    std::vector<lpa_graph *> graphs;
    GraphDev *gd = nullptr;
    size_t gd_cap = 0;
    RunState *rs = nullptr;
    size_t rs_cap = 0;
    WorkItem *items = nullptr;
    size_t items_cap = 0;
    unsigned *queues = nullptr;
    int32_t *active = nullptr;
    RunState *rs_h = nullptr;          // pinned mirror
    size_t rs_h_cap = 0;
    int32_t *active_h = nullptr;       // pinned
    SweepPlan plan{};

    ~MultiPlan()
    {
        if (gd) cudaFree(gd);
        if (rs) cudaFree(rs);
        if (items) cudaFree(items);
        if (queues) cudaFree(queues);
        if (active) cudaFree(active);
        if (rs_h) cudaFreeHost(rs_h);
        if (active_h) cudaFreeHost(active_h);
    }

    int ensure_host(size_t n)
    {
        if (!active_h && cudaMallocHost((void **)&active_h, sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            active_h = nullptr;
            set_error("cudaMallocHost failed");
            return LPA_ENOMEM;
        }
        if (n <= rs_h_cap && rs_h) return LPA_OK;
        if (rs_h) cudaFreeHost(rs_h);
        rs_h = nullptr;
        rs_h_cap = 0;
        const size_t c = std::max<size_t>(n, 16) * 3 / 2;
        if (cudaMallocHost((void **)&rs_h, c * sizeof(RunState)) != cudaSuccess) {
            cudaGetLastError();
            rs_h = nullptr;
            set_error("cudaMallocHost failed");
            return LPA_ENOMEM;
        }
        rs_h_cap = c;
        return LPA_OK;
    }

    // Builds the plan of `gs` (all with the same tuning); graph i's run state is rs[i].
    int build(const std::vector<lpa_graph *> &gs, const lpa_tuning &t)
    {
        graphs = gs;
        const size_t n = gs.size();
        LPA_CHECK(grow(&gd, &gd_cap, n));
        LPA_CHECK(grow(&rs, &rs_cap, n));
        LPA_CHECK(ensure_host(n));
        if (!queues && cudaMalloc((void **)&queues, sizeof(unsigned) * kQueueCount) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc failed");
            return LPA_ENOMEM;
        }
        if (!active && cudaMalloc((void **)&active, sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            set_error("cudaMalloc failed");
            return LPA_ENOMEM;
        }
        std::vector<GraphDev> gdh(n);
        bool all_int = true;
        for (size_t i = 0; i < n; ++i) {
            gdh[i] = gs[i]->gdh;
            gdh[i].rs = rs + i;
            all_int = all_int && plan_int_weights(gs[i]);
        }
        std::vector<WorkItem> all;
        size_t at[B_COUNT] = {}, at_h[HL_COUNT] = {}, at_pg;
        SweepPlan p{};
        for (int b = B_THREAD; b <= B_CTA_XL; ++b) {
            at[b] = all.size();
            for (size_t i = 0; i < n; ++i) {
                for (WorkItem it : gs[i]->items_h[b]) {
                    it.g = (int32_t)i;
                    all.push_back(it);
                }
                p.n_vertices[b] += gs[i]->bucket_start[b + 1] - gs[i]->bucket_start[b];
            }
            p.n_items[b] = (int32_t)(all.size() - at[b]);
        }
        for (int q = 0; q < HL_COUNT; ++q) {
            at_h[q] = all.size();
            for (size_t i = 0; i < n; ++i)
                for (WorkItem it : gs[i]->hub_items_h[q]) {
                    it.g = (int32_t)i;
                    all.push_back(it);
                }
            p.n_hub_items[q] = (int32_t)(all.size() - at_h[q]);
        }
        at_pg = all.size();
        for (size_t i = 0; i < n; ++i) all.push_back(WorkItem{(int32_t)i, 0, 0, 0});
        LPA_CHECK(grow(&items, &items_cap, all.size()));
        LPA_CUDA(cudaMemcpyAsync(gd, gdh.data(), n * sizeof(GraphDev), cudaMemcpyHostToDevice, stream));
        LPA_CUDA(cudaMemcpyAsync(items, all.data(), all.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, stream));
        LPA_CUDA(cudaStreamSynchronize(stream));      // the host vectors go out of scope
        p.gd = gd;
        p.n_graphs = (int32_t)n;
        for (int b = B_THREAD; b <= B_CTA_XL; ++b) p.items[b] = items + at[b];
        plan_slots(t, p.slots);
        for (int q = 0; q < HL_COUNT; ++q) p.hub_items[q] = items + at_h[q];
        p.per_graph = items + at_pg;
        p.queues = queues;
        p.active_count = active;
        p.group_lanes = t.group_lanes;
        p.flat_buckets = t.flat_buckets;
        p.cta_threads = t.cta_threads;
        p.cta_large_threads = t.cta_large_threads;
        p.cta_xl_threads = t.cta_xl_threads;
        p.hub_chunk = t.hub_chunk;
        p.int_weights = all_int ? 1 : 0;
        p.probe = t.probe;
        p.f64 = t.float_values == 2 ? 1 : 0;
        plan = p;
        return LPA_OK;
    }

    int upload_states(size_t n)
    {
        int32_t act = 0;
        for (size_t i = 0; i < n; ++i) act += rs_h[i].done ? 0 : 1;
        *active_h = act;
        LPA_CUDA(cudaMemcpyAsync(rs, rs_h, n * sizeof(RunState), cudaMemcpyHostToDevice, stream));
        LPA_CUDA(cudaMemcpyAsync(active, active_h, sizeof(int32_t), cudaMemcpyHostToDevice, stream));
        return LPA_OK;
    }

    int download_states(size_t n)
    {
        LPA_CUDA(cudaMemcpyAsync(rs_h, rs, n * sizeof(RunState), cudaMemcpyDeviceToHost, stream));
        LPA_CUDA(cudaStreamSynchronize(stream));
        return LPA_OK;
    }
};

RunState fresh_state(int64_t n, double tol, int max_iters, int pl_period, bool async_mode)
{
    RunState r{};
    r.l = 0;
    r.first = 0;
    r.max_iters = max_iters;
    r.pl_period = pl_period;
    r.async_mode = async_mode ? 1 : 0;
    r.mark = async_mode ? 1 : 0;                    // see lpa_run: a fresh synchronous run starts without marks
    r.tol = tol;
    r.n = n;
    r.fresh = 1;
    r.adaptive = 0;                                 // one kernel variant per sweep of a shared plan
    r.done = (n == 0 || max_iters <= 0) ? 1 : 0;
    return r;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

lpa_tuning multi_tuning()
{
    lpa_tuning t{};
    t.thread_max = 7;
    t.group_max = 31;
    t.group_lanes = 8;
    t.warp_max = 255;
    t.cta_max = 1023;
    t.cta_threads = 128;
    t.cta_large_max = 4095;
    t.cta_large_threads = 512;
    t.cta_xl_max = 8191;
    t.cta_xl_threads = 1024;
    t.hub_chunk = 16384;
    t.hub_table_shift = 1;
    t.smem_table_shift = 1;
    t.probe = 4;                                      // quadratic-double over power-of-two tables
    t.flat_buckets = 0;                               // one thread / lane group / warp per vertex
    t.hub_two_pass = 1;                               // hubs in two passes in a run's first sweep
    return t;
}

}  // namespace

// =======================================================================================
// batches

struct lpa_batch {
    int device = 0;
    cudaStream_t stream = nullptr;       // own non-blocking stream (graph capture)
    cudaStream_t user_stream = nullptr;
    Arena *arena = nullptr;
    std::vector<lpa_graph *> graphs;
    lpa_tuning tuning{};
    MultiPlan mp;
    cudaGraphExec_t exec = nullptr;
    int exec_span = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool built = false;
    unsigned long long *h_macc = nullptr;  // pinned: four modularity words per graph
};

static void batch_free(lpa_batch *b)
{
    if (!b) return;
    DeviceGuard dg(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (lpa_graph *g : b->graphs) destroy_graph(g, true);      // the arena goes below
    b->graphs.clear();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b->arena;
    b->arena = nullptr;
    if (b->h_macc) cudaFreeHost(b->h_macc);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;                                          // frees the plan arrays
}

// Runs fn(k, stream) for k = 0..count-1 on up to kHostThreads host threads, each with its own
// non-blocking stream (ordered after the batch stream's work so far) and the batch's device;
// every stream is synchronised before returning.  Returns the first failure's status, with
// its message in *msg (graph index k + index_base).
constexpr int kHostThreads = 8;

template <class Fn>
static int for_graphs_in_parallel(lpa_batch *b, int count, Fn fn, std::string *msg, int index_base)
{
    if (count <= 0) return LPA_OK;
    unsigned hc = std::thread::hardware_concurrency();
    const int threads = std::max(1, std::min<int>({kHostThreads, count, hc ? (int)hc : 1}));
    cudaEvent_t after = nullptr;
    if (cudaEventCreateWithFlags(&after, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        *msg = "event creation failed";
        return LPA_ECUDA;
    }
    cudaEventRecord(after, b->stream);
    std::atomic<int> next{0};
    std::atomic<int> status{LPA_OK};
    std::mutex mu;
    auto worker = [&]() {
        cudaSetDevice(b->device);
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            std::lock_guard<std::mutex> lock(mu);
            if (status.load() == LPA_OK) {
                status = LPA_ECUDA;
                *msg = "stream creation failed";
            }
            return;
        }
        cudaStreamWaitEvent(s, after, 0);
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= count || status.load() != LPA_OK) break;
            const int st = fn(k, s);
            if (st != LPA_OK) {
                std::lock_guard<std::mutex> lock(mu);
                if (status.load() == LPA_OK) {
                    status = st;
                    *msg = std::string(lpa_last_error()) + " (graph " + std::to_string(k + index_base) + ")";
                }
                break;
            }
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(worker);     // and this thread
    worker();
    for (std::thread &t : pool) t.join();
    cudaEventDestroy(after);
    return status.load();
}

extern "C" {

int lpa_batch_create(int n_graphs, const lpa_graph_desc *descs, int flags, void *cuda_stream, lpa_batch **out)
{
    if (!out || n_graphs < 1 || n_graphs > 65535 || !descs) {
        set_error("lpa_batch_create: need 1..65535 graphs and an output pointer");
        return LPA_EINVAL;
    }
    *out = nullptr;
    lpa_batch *b = new lpa_batch();
    cudaGetDevice(&b->device);
    b->user_stream = (cudaStream_t)cuda_stream;
    b->tuning = multi_tuning();
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        set_error("lpa_batch_create: stream or event creation failed");
        return LPA_ECUDA;
    }
    // the inputs may come from work ordered on the caller's stream
    cudaEvent_t ready;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(ready, b->user_stream);
        cudaStreamWaitEvent(b->stream, ready, 0);
        cudaEventDestroy(ready);
    }
    // arena: the inputs and per-vertex arrays up front, growth for tables and counters
    size_t est = 0;
    const bool i64 = (flags & LPA_OFFSETS_I64) != 0;
    for (int i = 0; i < n_graphs; ++i) {
        const lpa_graph_desc &d = descs[i];
        est += (size_t)(d.n_vertices + 1) * 8 + (size_t)d.n_entries * (d.weights ? 8 : 4) +
               (size_t)d.n_vertices * 22 + 16384;
        (void)i64;
    }
    b->arena = new Arena(est + (est >> 3) + ((size_t)64 << 20), true);
    if (!b->arena->ok()) {
        batch_free(b);
        set_error("lpa_batch_create: arena reservation failed");
        return LPA_ENOMEM;
    }
    b->mp.stream = b->stream;
    b->graphs.assign((size_t)n_graphs, nullptr);
    auto create_one = [&](int i, cudaStream_t s) {
        const lpa_graph_desc &d = descs[i];
        return create_graph(d.offsets, d.indices, d.weights, d.n_vertices, d.n_entries, flags, s, b->arena,
                            &b->tuning, &b->graphs[(size_t)i]);
    };
    // The first graph on this thread (it also settles the device properties computed on first
    // use); the others on several host threads, each with its own stream: creating a graph
    // waits on the device a few times (validation, weight properties, bucket sizes), and the
    // waits of different graphs then overlap.
    int st = create_one(0, b->stream);
    std::string msg = st == LPA_OK ? std::string() : std::string(lpa_last_error()) + " (graph 0)";
    if (st == LPA_OK && n_graphs > 1) {
        dsm_max_class_bits();
        st = for_graphs_in_parallel(b, n_graphs - 1, [&](int k, cudaStream_t s) { return create_one(k + 1, s); }, &msg,
                                    1);
    }
    for (lpa_graph *g : b->graphs)
        if (g) g->stream = b->stream;
    if (st != LPA_OK) {
        batch_free(b);
        set_error(msg);
        return st;
    }
    *out = b;
    return LPA_OK;
}

int lpa_batch_run(lpa_batch *b, double tolerance, int max_iters, int pl_period, int mode, lpa_result *results,
                  float *device_ms)
{
    if (!b || max_iters < 0 || pl_period < 0 || !std::isfinite(tolerance) || (mode != LPA_SYNC && mode != LPA_ASYNC)) {
        set_error("lpa_batch_run: bad arguments (mode must be LPA_SYNC or LPA_ASYNC)");
        return LPA_EINVAL;
    }
    DeviceGuard dg(b->device);
    const bool async_mode = mode == LPA_ASYNC;
    const size_t n = b->graphs.size();
    const int span = std::max(max_iters, 1);
    for (lpa_graph *g : b->graphs) {
        LPA_CHECK(ensure_counters(g, span, false));
        LPA_CHECK(upload_descriptor(g));
    }
    const GraphDev *gd_before = b->mp.gd;
    const WorkItem *items_before = b->mp.items;
    LPA_CHECK(b->mp.build(b->graphs, b->tuning));
    if (b->exec && (b->mp.gd != gd_before || b->mp.items != items_before)) {   // recorded pointers moved
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    for (size_t i = 0; i < n; ++i)
        b->mp.rs_h[i] = fresh_state(b->graphs[i]->n, tolerance, max_iters, pl_period, async_mode);
    LPA_CHECK(b->mp.upload_states(n));
    k_init_multi<<<dim3(4, (unsigned)n), 256, 0, b->stream>>>(b->mp.gd);
    LPA_CUDA(cudaGetLastError());
    if (b->exec && b->exec_span != span) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    // record the span sweeps once; replay them on every run (the plan arrays keep their
    // device addresses while the batch is unchanged)
    if (!b->exec) {
        cudaGraph_t graph = nullptr;
        LPA_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed));
        cudaError_t e = cudaSuccess;
        // Every run of a batch starts fresh at sweep 0, and only sweep 1 of a fresh synchronous
        // run takes its active vertices from moved bits (the run states are not adaptive):
        // that sweep launches both kernel variants (asynchronous runs replay the same
        // recording and use the push variant).
        for (int it = 0; it < span && e == cudaSuccess; ++it) {
            SweepPlan p = b->mp.plan;
            p.pull_mode = it == 1 ? 2 : 0;
            e = enqueue_sweep(p, b->stream, nullptr, nullptr);
        }
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            set_error(std::string("lpa_batch_run: graph capture: ") +
                      cudaGetErrorString(e != cudaSuccess ? e : e2));
            return LPA_ECUDA;
        }
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            set_error(std::string("lpa_batch_run: graph instantiation: ") + cudaGetErrorString(e));
            return LPA_ECUDA;
        }
        b->exec_span = span;
    }
    LPA_CUDA(cudaEventRecord(b->ev0, b->stream));
    LPA_CUDA(cudaGraphLaunch(b->exec, b->stream));
    LPA_CUDA(cudaEventRecord(b->ev1, b->stream));
    LPA_CHECK(b->mp.download_states(n));
    if (device_ms) cudaEventElapsedTime(device_ms, b->ev0, b->ev1);
    for (size_t i = 0; i < n; ++i) {
        const RunState &r = b->mp.rs_h[i];
        lpa_graph *g = b->graphs[i];
        g->next_iter = r.l;
        g->active_buf = async_mode ? 0 : (r.l & 1);
        if (results) {
            results[i].iterations = r.l;
            results[i].converged = r.converged;
            results[i].last_changed = r.last_dn;
        }
    }
    return LPA_OK;
}

int lpa_batch_labels(const lpa_batch *b, int graph, int32_t *out, int64_t n, int out_on_device)
{
    if (!b || graph < 0 || graph >= (int)b->graphs.size()) {
        set_error("lpa_batch_labels: bad graph index");
        return LPA_EINVAL;
    }
    return lpa_labels(b->graphs[graph], out, n, out_on_device);
}

int lpa_batch_modularity(lpa_batch *b, double *q)
{
    if (!b || !q) return LPA_EINVAL;
    DeviceGuard dg(b->device);
    const size_t n = b->graphs.size();
    if (!b->h_macc && cudaMallocHost((void **)&b->h_macc, n * 4 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        b->h_macc = nullptr;
        set_error("lpa_batch_modularity: cudaMallocHost failed");
        return LPA_ENOMEM;
    }
    // every graph's kernels and the copy of its four words on the batch stream, one wait at the
    // end (launches from several host threads measured slower: they contend for the context)
    for (size_t i = 0; i < n; ++i) {
        lpa_graph *g = b->graphs[i];
        LPA_CHECK(graph_modularity_enqueue(g));
        if (g->n > 0)
            LPA_CUDA(cudaMemcpyAsync(b->h_macc + 4 * i, g->macc, 4 * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, b->stream));
    }
    LPA_CUDA(cudaStreamSynchronize(b->stream));
    for (size_t i = 0; i < n; ++i) q[i] = graph_modularity_finish(b->graphs[i], b->h_macc + 4 * i);
    return LPA_OK;
}

int lpa_batch_graph(lpa_batch *b, int graph, lpa_graph **out)
{
    if (!b || !out || graph < 0 || graph >= (int)b->graphs.size()) {
        set_error("lpa_batch_graph: bad graph index");
        return LPA_EINVAL;
    }
    *out = b->graphs[graph];
    return LPA_OK;
}

int lpa_batch_get_tuning(const lpa_batch *b, lpa_tuning *t)
{
    if (!b || !t) return LPA_EINVAL;
    *t = b->tuning;
    return LPA_OK;
}

int lpa_batch_set_tuning(lpa_batch *b, const lpa_tuning *t)
{
    if (!b || !t) return LPA_EINVAL;
    DeviceGuard dg(b->device);
    LPA_CUDA(cudaStreamSynchronize(b->stream));
    const lpa_tuning old = b->tuning;
    for (size_t i = 0; i < b->graphs.size(); ++i) {
        const int st = lpa_set_tuning(b->graphs[i], t);
        if (st != LPA_OK) {                            // the first graph rejects an invalid tuning
            for (size_t j = 0; j < i; ++j) lpa_set_tuning(b->graphs[j], &old);
            return st;
        }
    }
    b->tuning = *t;
    if (b->exec) {                                     // launch shapes are recorded in the graph
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return LPA_OK;
}

int lpa_batch_size(const lpa_batch *b) { return b ? (int)b->graphs.size() : -1; }

int64_t lpa_batch_device_bytes(const lpa_batch *b) { return b ? (int64_t)b->arena->capacity() : -1; }

void lpa_batch_destroy(lpa_batch *b) { batch_free(b); }

}  // extern "C"

// =======================================================================================
// server

namespace {

struct Request {
    int64_t id = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> idx;
    std::vector<float> w;
    bool has_w = false;
    const void *b_off = nullptr;       // borrowed inputs (LPA_BORROW_INPUTS)
    const int32_t *b_idx = nullptr;
    const float *b_w = nullptr;
    int b_flags = 0;
    int64_t n = 0, m = 0;
    double tol = 0.0;
    int max_iters = 0, pl_period = 0;
    bool async_mode = false;
    double t_submit = 0.0, t_admit = 0.0, t_finish = 0.0;
    lpa_graph *g = nullptr;
    RunState rs{};
    std::vector<int32_t> labels;
    lpa_result res{};
    int status = LPA_OK;
};

}  // namespace

struct lpa_server {
    int device = 0;
    cudaStream_t stream = nullptr;       // own non-blocking stream
    Arena *arena = nullptr;
    int max_resident = 0;
    lpa_tuning tuning{};
    std::deque<Request *> queue;
    std::vector<Request *> running;
    std::map<int64_t, Request *> finished;
    int64_t next_id = 1;
    MultiPlan mp;
    bool dirty = true;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Starts a fresh run of an admitted request: labels = ids, flags, counters (k_init_multi on
// the request's own one-graph descriptor, whose run state is the handle's).
int start_request(lpa_server *s, Request *r)
{
    lpa_graph *g = r->g;
    LPA_CHECK(ensure_counters(g, std::max(r->max_iters, 1), false));
    r->rs = fresh_state(g->n, r->tol, r->max_iters, r->pl_period, r->async_mode);
    LPA_CHECK(upload_descriptor(g));
    LPA_CUDA(cudaMemcpyAsync(g->rs_d, &r->rs, sizeof(RunState), cudaMemcpyHostToDevice, s->stream));
    k_init_multi<<<dim3(8, 1), 256, 0, s->stream>>>(g->gdd);
    LPA_CUDA(cudaGetLastError());
    LPA_CUDA(cudaStreamSynchronize(s->stream));
    return LPA_OK;
}

void finish_request(lpa_server *s, Request *r, int status)
{
    r->status = status;
    r->t_finish = s->now();
    if (r->g) {
        if (status == LPA_OK && r->g->n > 0) {
            r->labels.resize((size_t)r->g->n);
            if (lpa_labels(r->g, r->labels.data(), r->g->n, 0) != LPA_OK) r->status = LPA_ECUDA;
        }
        destroy_graph(r->g);
        r->g = nullptr;
    }
    r->res.iterations = r->rs.l;
    r->res.converged = r->rs.converged;
    r->res.last_changed = r->rs.last_dn;
    s->finished[r->id] = r;
}

}  // namespace

extern "C" {

int lpa_server_create(size_t hbm_budget_bytes, int max_resident, void *cuda_stream, lpa_server **out)
{
    (void)cuda_stream;
    if (!out || hbm_budget_bytes < ((size_t)1 << 20) || max_resident < 1 || max_resident > 65535) {
        set_error("lpa_server_create: budget of at least 1 MiB and 1..65535 resident requests");
        return LPA_EINVAL;
    }
    *out = nullptr;
    lpa_server *s = new lpa_server();
    cudaGetDevice(&s->device);
    s->max_resident = max_resident;
    s->tuning = multi_tuning();
    s->t0 = std::chrono::steady_clock::now();
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        set_error("lpa_server_create: stream creation failed");
        return LPA_ECUDA;
    }
    s->mp.stream = s->stream;
    s->arena = new Arena(hbm_budget_bytes, false);
    if (!s->arena->ok()) {
        cudaStreamDestroy(s->stream);
        delete s->arena;
        delete s;
        set_error("lpa_server_create: could not reserve the HBM budget");
        return LPA_ENOMEM;
    }
    *out = s;
    return LPA_OK;
}

int lpa_server_submit(lpa_server *s, const lpa_graph_desc *graph, int flags, double tolerance, int max_iters,
                      int pl_period, int mode, int64_t *request_id)
{
    if (!s || !graph || !request_id || graph->n_vertices < 0 || graph->n_entries < 0 || !graph->offsets ||
        (graph->n_entries > 0 && !graph->indices) || max_iters < 0 || pl_period < 0 || !std::isfinite(tolerance) ||
        (mode != LPA_SYNC && mode != LPA_ASYNC) || (flags & LPA_DEVICE_PTRS)) {
        set_error("lpa_server_submit: bad arguments (host arrays, mode LPA_SYNC or LPA_ASYNC)");
        return LPA_EINVAL;
    }
    const int64_t n = graph->n_vertices, m = graph->n_entries;
    // lower bound of the resident footprint: CSR, labels, two flag arrays, mover lists, buckets
    const size_t need = (size_t)(n + 1) * 8 + (size_t)m * (graph->weights ? 8 : 4) + (size_t)n * 22;
    if (need > s->arena->capacity()) {
        set_error("lpa_server_submit: the graph can never fit the server's HBM budget");
        return LPA_EINVAL;
    }
    Request *r = new Request();
    r->n = n;
    r->m = m;
    if (flags & LPA_BORROW_INPUTS) {
        r->b_off = graph->offsets;
        r->b_idx = graph->indices;
        r->b_w = graph->weights;
        r->b_flags = flags & LPA_OFFSETS_I64;
    } else {
        r->off.resize((size_t)n + 1);
        if (flags & LPA_OFFSETS_I64) {
            memcpy(r->off.data(), graph->offsets, ((size_t)n + 1) * sizeof(int64_t));
        } else {
            const int32_t *o = static_cast<const int32_t *>(graph->offsets);
            for (int64_t i = 0; i <= n; ++i) r->off[(size_t)i] = o[i];
        }
        r->idx.assign(graph->indices, graph->indices + m);
        if (graph->weights) {
            r->has_w = true;
            r->w.assign(graph->weights, graph->weights + m);
        }
    }
    r->tol = tolerance;
    r->max_iters = max_iters;
    r->pl_period = pl_period;
    r->async_mode = mode == LPA_ASYNC;
    std::lock_guard<std::mutex> lock(s->mu);
    r->id = s->next_id++;
    r->t_submit = s->now();
    s->queue.push_back(r);
    *request_id = r->id;
    return LPA_OK;
}

int lpa_server_step(lpa_server *s, int *n_completed, int *n_running, int *n_queued)
{
    if (!s) return LPA_EINVAL;
    DeviceGuard dg(s->device);
    std::lock_guard<std::mutex> lock(s->mu);
    int completed = 0;
    // admission: arrival order, later requests may pass one that does not fit yet
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)s->running.size() < s->max_resident;) {
        Request *r = *it;
        lpa_graph *g = nullptr;
        const int st = r->b_off
            ? create_graph(r->b_off, r->b_idx, r->b_w, r->n, r->m, r->b_flags | LPA_HOST_PTRS, s->stream, s->arena,
                           &s->tuning, &g)
            : create_graph(r->off.data(), r->idx.data(), r->has_w ? r->w.data() : nullptr, r->n, r->m,
                           LPA_OFFSETS_I64 | LPA_HOST_PTRS, s->stream, s->arena, &s->tuning, &g);
        if (st == LPA_ENOMEM && !s->running.empty()) {
            ++it;                                      // waits for memory to free up
            continue;
        }
        if (st != LPA_OK) {                            // invalid, or too large even alone
            it = s->queue.erase(it);
            finish_request(s, r, st);
            ++completed;
            continue;
        }
        r->g = g;
        const int st2 = start_request(s, r);
        if (st2 != LPA_OK) {
            it = s->queue.erase(it);
            finish_request(s, r, st2);
            ++completed;
            continue;
        }
        r->t_admit = s->now();
        r->off = std::vector<int64_t>();
        r->idx = std::vector<int32_t>();
        r->w = std::vector<float>();
        s->running.push_back(r);
        it = s->queue.erase(it);
        s->dirty = true;
    }
    if (!s->running.empty()) {
        const size_t n = s->running.size();
        if (s->dirty) {
            std::vector<lpa_graph *> gs;
            for (Request *r : s->running) gs.push_back(r->g);
            for (lpa_graph *g : gs) LPA_CHECK(upload_descriptor(g));
            LPA_CHECK(s->mp.build(gs, s->tuning));
            s->dirty = false;
        }
        bool any_pull = false, any_push = false;
        for (size_t i = 0; i < n; ++i) {
            s->mp.rs_h[i] = s->running[i]->rs;
            (s->running[i]->rs.pull ? any_pull : any_push) = true;
        }
        LPA_CHECK(s->mp.upload_states(n));
        s->mp.plan.pull_mode = any_pull ? (any_push ? 2 : 1) : 0;
        LPA_CUDA(enqueue_sweep(s->mp.plan, s->stream, nullptr, nullptr));
        LPA_CHECK(s->mp.download_states(n));
        std::vector<Request *> still;
        for (size_t i = 0; i < n; ++i) {
            Request *r = s->running[i];
            r->rs = s->mp.rs_h[i];
            if (r->rs.done) {
                r->g->next_iter = r->rs.l;
                r->g->active_buf = r->async_mode ? 0 : (r->rs.l & 1);
                finish_request(s, r, LPA_OK);
                ++completed;
                s->dirty = true;
            } else {
                still.push_back(r);
            }
        }
        s->running.swap(still);
    }
    if (n_completed) *n_completed = completed;
    if (n_running) *n_running = (int)s->running.size();
    if (n_queued) *n_queued = (int)s->queue.size();
    return LPA_OK;
}

int lpa_server_cancel(lpa_server *s, int64_t request_id)
{
    if (!s) return LPA_EINVAL;
    DeviceGuard dg(s->device);
    std::lock_guard<std::mutex> lock(s->mu);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        if ((*it)->id != request_id) continue;
        Request *r = *it;
        s->queue.erase(it);
        finish_request(s, r, LPA_ECANCELED);
        return LPA_OK;
    }
    // between steps no work of the server is in flight (a step ends by synchronising)
    for (size_t i = 0; i < s->running.size(); ++i) {
        if (s->running[i]->id != request_id) continue;
        Request *r = s->running[i];
        s->running.erase(s->running.begin() + (long)i);
        finish_request(s, r, LPA_ECANCELED);
        s->dirty = true;
        return LPA_OK;
    }
    if (s->finished.count(request_id)) {
        set_error("lpa_server_cancel: the request has finished");
        return LPA_ESTATE;
    }
    set_error("lpa_server_cancel: unknown request");
    return LPA_EINVAL;
}

int lpa_server_poll(lpa_server *s, int64_t *ids, int max_ids, int *n)
{
    if (!s || !n || (max_ids > 0 && !ids)) return LPA_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    int k = 0;
    for (const auto &kv : s->finished) {
        if (k >= max_ids) break;
        ids[k++] = kv.first;
    }
    *n = k;
    return LPA_OK;
}

int lpa_server_result(lpa_server *s, int64_t request_id, int32_t *labels, int64_t n, lpa_result *result,
                      double *t_submit, double *t_admit, double *t_finish)
{
    if (!s) return LPA_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->finished.find(request_id);
    if (it == s->finished.end()) {
        set_error("lpa_server_result: request not finished (or unknown)");
        return LPA_ESTATE;
    }
    Request *r = it->second;
    if (labels) {
        if (n != r->n) {
            set_error("lpa_server_result: n does not match the request's vertex count");
            return LPA_EINVAL;
        }
        if (!r->labels.empty()) memcpy(labels, r->labels.data(), (size_t)n * sizeof(int32_t));
    }
    if (result) *result = r->res;
    if (t_submit) *t_submit = r->t_submit;
    if (t_admit) *t_admit = r->t_admit;
    if (t_finish) *t_finish = r->t_finish;
    const int st = r->status;
    s->finished.erase(it);
    delete r;
    return st;
}

double lpa_server_clock(const lpa_server *s) { return s ? s->now() : 0.0; }

int64_t lpa_server_device_bytes(const lpa_server *s) { return s ? (int64_t)s->arena->used() : -1; }

void lpa_server_destroy(lpa_server *s)
{
    if (!s) return;
    DeviceGuard dg(s->device);
    cudaStreamSynchronize(s->stream);
    for (Request *r : s->running) {
        if (r->g) destroy_graph(r->g);
        delete r;
    }
    for (Request *r : s->queue) delete r;
    for (auto &kv : s->finished) delete kv.second;
    delete s->arena;
    s->arena = nullptr;
    cudaStreamDestroy(s->stream);
    delete s;                                          // frees the plan arrays
}

}  // extern "C"
