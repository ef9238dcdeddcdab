// The graph handle and the helpers shared by lpa_graph.cu (single graphs) and lpa_multi.cu
// (batches and the server).
#pragma once

#include <utility>
#include <vector>

#include "lpa_internal.h"

struct lpa_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    lpa::Arena *arena = nullptr;                     // device blocks come from here when set
    std::vector<std::pair<void *, size_t>> allocs;   // owned device blocks
    int64_t n = 0, m = 0;
    int64_t *off = nullptr;
    int32_t *idx = nullptr;
    float *w = nullptr;
    int32_t *C = nullptr;
    uint8_t *flags[2] = {nullptr, nullptr};
    int active_buf = 0;                              // flags[active_buf]: unprocessed flags of the next sweep
    int32_t *mover_v = nullptr, *mover_v1 = nullptr, *mover_c = nullptr;
    int32_t *cc_prev = nullptr, *cc_midx = nullptr, *cc_par0 = nullptr;   // Cross-Check (on demand)
    long long *cc_word = nullptr;
    unsigned *cc_ctr = nullptr;
    unsigned long long *mover_count = nullptr;       // [2]
    unsigned long long *fallbacks = nullptr;
    unsigned long long *ctr = nullptr;               // [ctr_iters][kPerSweep]
    int ctr_iters = 0;
    unsigned long long *h_ctr = nullptr;             // pinned mirror for lpa_run statistics
    int h_ctr_iters = 0;
    unsigned *d_err = nullptr;
    double *Sig = nullptr, *macc = nullptr;
    lpa_tuning tuning{};
    int32_t *lists = nullptr;
    int64_t bucket_start[lpa::B_COUNT + 1] = {};
    // hubs
    void *hub_mem = nullptr;
    int32_t *tab_k = nullptr;
    float *tab_v = nullptr;
    int32_t *used_list = nullptr;
    unsigned long long *pairs = nullptr;             // two-pass hub partitions: [n_parts * kPartCap]
    int64_t table_slots = 0;
    // work items of this graph (graph index 0); batches re-index copies of the host vectors
    std::vector<lpa::WorkItem> items_h[lpa::B_COUNT];
    std::vector<lpa::WorkItem> hub_items_h[lpa::HL_COUNT];
    lpa::WorkItem *items_d = nullptr;                // every item of this graph in one block
    lpa::WorkItem *items_at[lpa::B_COUNT] = {};
    lpa::WorkItem *hub_items_d[lpa::HL_COUNT] = {};
    lpa::WorkItem *per_graph_d = nullptr;
    // descriptor and run state of this graph alone (lpa_run)
    lpa::GraphDev gdh{};
    lpa::GraphDev *gdd = nullptr;
    lpa::RunState *rs_d = nullptr;
    unsigned *queues = nullptr;
    int32_t *active = nullptr;
    struct HostMirror {
        lpa::RunState rs;
        int32_t active;
        int32_t pad;
    } *hm = nullptr;                                 // pinned
    int next_iter = 0;
    bool int_weights = false;                        // integer weights, weighted degrees < 2^24
    bool rows_strict = false;                        // every row's indices strictly increase
    int64_t bytes = 0;
    std::vector<cudaEvent_t> events;
};

namespace lpa {

// Creates a graph handle; device blocks come from `arena` when it is not null.
int create_graph(const void *offsets, const int32_t *indices, const float *weights, int64_t n_vertices,
                 int64_t n_entries, int flags, cudaStream_t stream, Arena *arena, const lpa_tuning *tuning,
                 lpa_graph **out);
// Frees a graph handle.  arena_released: the caller has synchronised the graph's stream and
// releases the whole arena the graph's blocks came from, so they are not returned one by one.
void destroy_graph(lpa_graph *g, bool arena_released = false);
// Counter rows for `iters` sweeps (device; the pinned mirror only when `mirror`).
int ensure_counters(lpa_graph *g, int iters, bool mirror);
// Smem slots per table of each vertex kernel for a tuning.
void plan_slots(const lpa_tuning &t, int32_t slots[B_COUNT]);
// Fills g->gdh from the handle (pointers, hub arrays, counters) and uploads it to g->gdd.
int upload_descriptor(lpa_graph *g);
bool plan_int_weights(const lpa_graph *g);
// Modularity of one graph (float64, or exact for integer weights).
int graph_modularity(lpa_graph *g, double *q);
// The same in two halves: enqueue the kernels that fill g->macc (four 8-byte words, on
// g->stream), then Q from a host copy of those words.
int graph_modularity_enqueue(lpa_graph *g);
double graph_modularity_finish(const lpa_graph *g, const void *acc_words);

}  // namespace lpa
