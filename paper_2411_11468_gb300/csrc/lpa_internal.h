// Internal definitions shared by the CUDA translation units of liblpa.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lpa.h"

namespace lpa {

constexpr int32_t kEmpty = -1;     // empty hashtable key (labels are >= 0)
constexpr int kMaxRetries = 32;    // hybrid probes before the linear fallback (Algorithm 2)
constexpr int kCtrFields = 4;      // per kernel slot: active, edges, moved, marks
enum { CTR_ACTIVE = 0, CTR_EDGES = 1, CTR_MOVED = 2, CTR_MARKS = 3 };
enum Bucket { B_THREAD = 0, B_GROUP, B_WARP, B_CTA, B_CTA_LARGE, B_CTA_XL, B_HUB, B_COUNT };

// Arguments of one sweep (Algorithm 1, lpaMove), passed by value to every sweep kernel.
struct SweepArgs {
    const int64_t *off;        // CSR offsets [n+1]
    const int32_t *idx;        // CSR neighbour ids [m]
    const float *w;            // CSR weights [m] or nullptr (unit)
    int32_t *C;                // labels [n]
    uint8_t *flag_cur;         // unprocessed flags read (and cleared) by this sweep
    uint8_t *flag_next;        // flags set for the next sweep (== flag_cur in ASYNC mode)
    int32_t *mover_v;          // SYNC: vertices that moved this sweep
    int32_t *mover_c;          // SYNC: their new labels
    unsigned long long *mover_count;
    unsigned long long *ctr;   // this sweep's counters [LPA_NUM_KERNELS][kCtrFields]
    unsigned long long *fallbacks;
    int32_t pl;                // Pick-Less active on this sweep
    int32_t async_mode;        // 1: write labels in place (ASYNC), 0: record movers (SYNC)
    int32_t tshift;            // smem table capacity = nextPow2(D << tshift) - 1
    int32_t persist_mask;      // bit k: kernel slot k runs as a persistent grid
    int32_t int_weights;       // 1: integer weights with weighted degrees < 2^24 (uint32 sums)
};

// Hub-bucket device arrays.
struct HubArgs {
    const int32_t *hub_v;      // [H] vertex of each hub
    const uint32_t *hub_p1;    // [H] table capacity (2^b - 1)
    const uint32_t *hub_b;     // [H] b
    const int64_t *hub_tab;    // [H] first slot of the hub's table
    uint8_t *hub_act;          // [H] this sweep: 0 processed earlier, 1 processing, 2 moved
    unsigned long long *hub_best;  // [H] packed (weight, ~label) maximum
    uint32_t *hub_used;        // [H] number of table slots taken this sweep
    int32_t *used_list;        // slots taken, hub h at used_base[h] (at most D_h entries)
    const int64_t *used_base;  // [H]
    const int32_t *chunk_h;    // [n_chunks] hub of each accumulate / mark block
    const int64_t *chunk_e0;   // [n_chunks] first CSR entry
    const int64_t *chunk_e1;   // [n_chunks] end CSR entry
    const int32_t *slice_h;    // [n_slices] hub of each argmax block
    const int32_t *slice_j;    // [n_slices] slice index within the hub's used list
    int32_t *tab_k;            // hub table keys
    float *tab_v;              // hub table values
    int32_t n_hubs;
};

constexpr int kHubSlice = 4096;   // used-list entries per argmax block

// Launch helpers implemented in lpa_sweep.cu.
cudaError_t sweep_init_constants();
cudaError_t launch_thread_bucket(const int32_t *list, int64_t count, const SweepArgs &a,
                                 int slots, cudaStream_t s);
cudaError_t launch_group_bucket(const int32_t *list, int64_t count, const SweepArgs &a, int lanes,
                                int slots, cudaStream_t s);
cudaError_t launch_warp_bucket(const int32_t *list, int64_t count, const SweepArgs &a, int slots,
                               cudaStream_t s);
cudaError_t launch_cta_bucket(const int32_t *list, int64_t count, const SweepArgs &a, int threads,
                              int slots, int kslot, cudaStream_t s);
cudaError_t launch_hub_begin(const HubArgs &h, const SweepArgs &a, cudaStream_t s);
cudaError_t launch_hub_acc(const HubArgs &h, const SweepArgs &a, int64_t n_chunks, int chunk, cudaStream_t s);
cudaError_t launch_hub_clear(const HubArgs &h, int64_t n_slices, cudaStream_t s);
cudaError_t launch_hub_move(const HubArgs &h, const SweepArgs &a, cudaStream_t s);
cudaError_t launch_hub_mark(const HubArgs &h, const SweepArgs &a, int64_t n_chunks, cudaStream_t s);
cudaError_t launch_apply(const SweepArgs &a, int64_t n, cudaStream_t s);
cudaError_t launch_hub_table_clear(int32_t *k, float *v, int64_t slots, cudaStream_t s);
size_t max_dynamic_smem();

// Thread-local error message.
void set_error(const std::string &msg);

}  // namespace lpa
