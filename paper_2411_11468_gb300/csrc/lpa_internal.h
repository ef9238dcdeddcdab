// Internal definitions shared by the CUDA translation units of liblpa.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lpa.h"

namespace lpa {

constexpr int32_t kEmpty = -1;     // empty hashtable key (labels are >= 0)
constexpr int kMaxRetries = 32;    // hybrid probes before the linear fallback (Algorithm 2)
constexpr int kCtrFields = 4;      // per kernel slot: active, edges, moved, marks
enum { CTR_ACTIVE = 0, CTR_EDGES = 1, CTR_MOVED = 2, CTR_MARKS = 3 };
enum Bucket { B_THREAD = 0, B_GROUP, B_WARP, B_CTA, B_CTA_LARGE, B_CTA_XL, B_HUB, B_COUNT };
// Work-item lists of the hub bucket: hubs (begin, move), accumulate chunks of hubs whose table
// is in HBM, mark chunks of every hub, clear slices of HBM tables, and the hubs whose table
// lives in the distributed shared memory of a 2-, 4-, 8- or 16-block cluster.
// Hubs with integer label sums and HBM tables take a two-pass accumulation instead: the
// chunks of the first pass (kPartChunk entries each) and the label partitions of the second.
enum HubList { HL_HUBS = 0, HL_ACC, HL_MARK, HL_SLICES, HL_DSM2, HL_DSM4, HL_DSM8, HL_DSM16, HL_PACC, HL_PMERGE,
               HL_COUNT };
// Two-pass hub accumulation: the first pass sums each kPartChunk-entry chunk of a hub's row in
// a shared-memory table and sends the chunk's distinct (label, sum) pairs to the hub's label
// partitions (2^pb of them, chosen so that a partition expects at most kPartExpect pairs when
// every label is distinct); the second pass sums each partition's pairs in a shared-memory
// table.  A partition holds at most kPartCap pairs; one that would overflow sends all its pairs
// to the hub's HBM table instead.
constexpr int kPartChunk = 4096;
constexpr int kPartExpect = 2048;
constexpr int kPartCap = 4096;
constexpr int kPartMaxBits = 10;
constexpr int kDsmSliceBits = 14;  // table slots per cluster block (2^14 x 8 bytes = 128 KB)
constexpr int kDsmMaxBits = 18;    // largest table in cluster shared memory: 2^18 slots over 16 blocks
// Work-queue counters: vertex buckets for push and pull launches, then the cluster classes.
constexpr int kQueueCount = 2 * B_COUNT + 2 * 4;
constexpr int kHubSlice = 4096;    // table slots / used-list entries per hub clear block
constexpr int kPerSweep = LPA_NUM_KERNELS * kCtrFields;   // counter words per sweep

// Run state of one graph, device-resident.  Sweep kernels read it; k_decide (after each
// sweep) applies the stop rule of Algorithm 1 and advances l.
struct RunState {
    int32_t l;            // absolute index of the sweep about to run
    int32_t first;        // absolute index of this run's first sweep (counter slot 0)
    int32_t max_iters;
    int32_t pl_period;
    int32_t async_mode;
    int32_t done;         // the run has stopped (tolerance or cap); no more work for this graph
    int32_t converged;    // stopped by the tolerance test
    int32_t mark;         // this sweep marks the neighbours of its movers (else movers get the moved bit)
    double tol;
    int64_t n;            // vertices (dN / n)
    int64_t last_dn;
    int32_t pull;         // this sweep takes activity from the previous sweep's moved bits
    int32_t fin;          // stopped after a sweep that set moved bits: k_finalize turns them into marks
    int32_t cc_period;    // Cross-Check after sweeps l with l mod cc_period = 0 (0: never; sync only)
    int32_t cc_unresolved;  // set when the Cross-Check resolution did not finish (not expected)
    int32_t fresh;        // the run started from labels = vertex ids (not resumed)
    int32_t adaptive;     // marks follow each sweep's moves (single-graph runs; else only sweep 1 pulls)
};

// Synchronous mode, sweeps that move many vertices: instead of marking the neighbours of each
// mover, the mover's label word gets bit 31 (labels are below 2^31), and the next sweep
// processes every vertex and takes as active those with a neighbour whose bit is set: the
// same active set as the marks give (a vertex is active iff a neighbour moved).
constexpr uint32_t kMovedBit = 0x80000000u;
constexpr uint32_t kLabelMask = 0x7FFFFFFFu;

// Hub-bucket device arrays of one graph.
struct HubArgs {
    const int32_t *hub_v;      // [H] vertex of each hub
    const uint32_t *hub_p1;    // [H] table capacity (2^b - 1)
    const uint32_t *hub_b;     // [H] b
    const int64_t *hub_tab;    // [H] first slot of the hub's table
    uint8_t *hub_act;          // [H] this sweep: 0 processed earlier, 1 processing, 2 moved
    uint8_t *hub_seen;         // [H] pull sweeps: a neighbour's moved bit was seen
    unsigned long long *hub_best;  // [H] packed (weight, ~label) maximum
    uint32_t *hub_used;        // [H] number of table slots taken this sweep
    int32_t *used_list;        // slots taken, hub h at used_base[h] (at most D_h entries)
    const int64_t *used_base;  // [H]
    const int32_t *chunk_h;    // [n_chunks] hub of each accumulate / mark block
    const int64_t *chunk_e0;   // [n_chunks] first CSR entry
    const int64_t *chunk_e1;   // [n_chunks] end CSR entry
    const int32_t *slice_h;    // [n_slices] hub of each clear block
    const int32_t *slice_j;    // [n_slices] slice index within the hub's table / used list
    int32_t *tab_k;            // hub tables: keys (split layout) or 64-bit slots over tab_k and tab_v (packed)
    float *tab_v;              // hub table values (split layout; directly after tab_k)
    double *tab_vd;            // float64 table values (lpa_tuning.float_values = 2), else null
    double *chunk_bv;          // float64 values: [n_chunks] arg-max pair of each accumulate
    int32_t *chunk_bk;         //   block (label < 0: none), reduced per hub by k_hub_move
    const int32_t *hub_c0;     // float64 values: [H + 1] first accumulate chunk of each hub
    // two-pass accumulation (integer sums, HBM tables)
    const int32_t *pc_h;       // [n_pchunks] hub of each first-pass chunk
    const int64_t *pc_e0;      // [n_pchunks] first CSR entry
    const int64_t *pc_e1;      // [n_pchunks] end CSR entry
    const uint32_t *hub_pb;    // [H] log2 of the hub's partitions
    const int32_t *hub_pbase;  // [H] first partition of the hub (-1: not two-pass)
    const int32_t *part_h;     // [n_parts] hub of each partition
    uint32_t *part_cnt;        // [n_parts] pairs sent to the partition this sweep
    int32_t *part_ovf;         // [n_parts] 1: the partition overflowed (pairs go to the HBM table)
    unsigned long long *pairs; // [n_parts * kPartCap] (label << 32 | sum)
    int32_t n_hubs;
    int32_t n_chunks;
    int32_t n_slices;
    int32_t pad;
};

// Static description of one resident graph, device-resident (an array of them per launch).
struct GraphDev {
    const int64_t *off;        // CSR offsets [n+1]
    const int32_t *idx;        // CSR neighbour ids [m]
    const float *w;            // CSR weights [m] or nullptr (unit)
    int32_t *C;                // labels [n]
    uint8_t *flags0, *flags1;  // processed flags; sweep l reads flags[l & 1] (sync) or flags0 (async)
    int32_t *mover_v;          // sync: vertices that moved in an even sweep
    int32_t *mover_v1;         // sync: vertices that moved in an odd sweep
    int32_t *mover_c;          // sync: new labels of this sweep's movers
    unsigned long long *mover_count;   // [2]: movers of the even / odd sweep
    unsigned long long *ctr;   // [ctr_iters][kPerSweep] per-sweep counters of this run
    unsigned long long *fallbacks;
    const int32_t *lists;      // degree-bucket vertex lists
    RunState *rs;
    int32_t ctr_iters;
    int32_t tshift;            // smem table capacity = nextPow2(D << tshift) - 1
    int32_t int_weights;       // integer weights with weighted degrees < 2^24 (uint32 sums)
    int32_t probe;             // table probe scheme (lpa_tuning.probe)
    int32_t hub_tp;            // two-pass hubs: 0 never, 1 in a run's first sweep, 2 every sweep
    int32_t hub_deg;           // rows longer than this are hubs (the hub bucket)
    int32_t rows_strict;       // every row's indices strictly increase (no repeated neighbour)
    int32_t pad_rs;
    // Cross-Check (allocated when a run asks for it): labels before the sweep of each mover,
    // vertex -> position in the mover list (-1 otherwise), per position the parent position
    // (or -1 / -2 for a move found good / bad directly) and the resolution word
    int32_t *cc_prev;
    int32_t *cc_midx;
    int32_t *cc_par0;
    long long *cc_word;
    HubArgs hub;
};

// A unit of work of one kernel kind: for vertex kernels, entries [start, start + count) of
// graph g's bucket list; for hub kernels, hubs / chunks / slices [start, start + count).
struct WorkItem {
    int32_t g;
    int32_t pad;
    int64_t start;
    int64_t count;
};

// One launch of every kernel of a sweep over a set of graphs (one graph for lpa_run, many
// for batches and the server).  Launch shapes are uniform over the set.
struct SweepPlan {
    const GraphDev *gd;        // device array of graph descriptors
    int32_t n_graphs;
    const WorkItem *items[B_COUNT];    // vertex items per bucket (B_HUB unused)
    int32_t n_items[B_COUNT];
    int64_t n_vertices[B_COUNT];       // vertices covered by the items of each bucket
    int32_t slots[B_COUNT];    // smem slots per table for each vertex kernel
    const WorkItem *hub_items[HL_COUNT];       // hub work items (HubList)
    int32_t n_hub_items[HL_COUNT];
    const WorkItem *per_graph;         // one item per graph (apply, decide)
    unsigned *queues;          // [kQueueCount] work-queue counters, zeroed per sweep
    int32_t *active_count;     // device counter written by k_decide (graphs still running)
    int32_t group_lanes, cta_threads, cta_large_threads, cta_xl_threads, hub_chunk;
    int32_t flat_buckets;      // bit b: bucket b (thread, group, warp) runs the flattened kernel
    int32_t pull_mode;         // kernels launched for this sweep: 0 push only, 1 pull only, 2 both
    int32_t int_weights;       // 1: every graph of the plan uses uint32 sums (else float32)
    int32_t probe;             // table probe scheme of every graph of the plan (lpa_tuning.probe)
    int32_t cc_any;            // some graph of the plan may run a Cross-Check (launch its kernels)
    int32_t f64;               // every graph of the plan keeps float64 table values
    unsigned *cc_ctr;          // [kCcPasses + 1] pending counts of the resolution passes
};

constexpr int kCcPasses = 40;      // pointer-jumping passes of the Cross-Check resolution (>= 32)

// Optional hook around each kernel launch (CUDA-event timing per kernel slot).
struct LaunchHook {
    virtual void before(int slot) = 0;
    virtual void after(int slot) = 0;
    virtual ~LaunchHook() {}
};

cudaError_t sweep_init_constants();
// Enqueues one sweep of every graph of the plan (graphs whose run has stopped do no work),
// the synchronous label publication and k_decide.  *launches counts kernel launches.
cudaError_t enqueue_sweep(const SweepPlan &p, cudaStream_t s, LaunchHook *hook, int *launches);
// Clears `slots` hub-table slots: packed (one 64-bit word per slot over k), split (k, v) or
// split with float64 values (k, vd; v unused).
cudaError_t launch_hub_table_clear(int32_t *k, float *v, int64_t slots, bool packed, cudaStream_t s,
                                   double *vd = nullptr);
size_t max_dynamic_smem();
// Largest cluster class (log2 of the blocks per cluster, 0 = none) that the device can run
// with a hub table slice of 2^kDsmSliceBits slots per block.
int dsm_max_class_bits();
int num_sms();

// Device memory arena: reservations carved into 256-byte aligned blocks (first fit with a
// coalescing free list).  Batches and the server allocate their graphs from it, so thousands
// of graphs do not each cost a dozen cudaMalloc calls, and a fixed arena turns admission by
// footprint into "the allocation fits".  A growing arena adds reservations on demand.
class Arena {
  public:
    Arena(size_t bytes, bool grow, size_t grow_chunk = (size_t)1 << 30);
    ~Arena();
    bool ok() const { return !regions_.empty(); }
    void *alloc(size_t bytes);
    void free(void *p);
    size_t capacity() const;
    size_t used() const;
    size_t largest_free() const;

  private:
    struct Region {
        unsigned char *base = nullptr;
        size_t cap = 0, used = 0;
        std::map<size_t, size_t> free_;  // offset -> size, coalesced
        std::map<size_t, size_t> taken_; // offset -> size
    };
    bool add_region(size_t bytes);
    static void *region_alloc(Region &r, size_t bytes);
    std::mutex mu_;                      // allocations from several host threads (batch creation)
    std::vector<Region> regions_;
    bool grow_ = false;
    size_t grow_chunk_ = 0;
};

// Thread-local error message.
void set_error(const std::string &msg);

}  // namespace lpa

// Early returns on a failed CUDA call (message recorded, status LPA_ENOMEM or LPA_ECUDA) or
// on a failed library status.
#define LPA_CUDA(call)                                                                       \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess) {                                                             \
            ::lpa::set_error(std::string(#call) + ": " + cudaGetErrorString(_e));            \
            return _e == cudaErrorMemoryAllocation ? LPA_ENOMEM : LPA_ECUDA;                 \
        }                                                                                    \
    } while (0)

#define LPA_CHECK(st)                                                                        \
    do {                                                                                     \
        int _s = (st);                                                                       \
        if (_s != LPA_OK) return _s;                                                         \
    } while (0)
