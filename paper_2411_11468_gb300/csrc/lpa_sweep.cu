// Sweep kernels of liblpa.so: one label-propagation sweep (Algorithm 1, lpaMove) over the
// vertices of one degree bucket, with per-vertex open-addressing hashtables probed by the
// hybrid quadratic-double sequence of Algorithm 2.
//
// Buckets (by degree D, thresholds in lpa_tuning):
//   thread      one thread per vertex, private table in shared memory (no atomics)
//   group       2..16 lanes per vertex, table in shared memory (shared-memory atomics)
//   warp        one warp per vertex, table in shared memory
//   cta tiers   one thread block per vertex (three block sizes), table in shared memory
//   hub         several blocks per vertex, table in HBM (global atomics)
// Table capacity is p1 = 2^b - 1 >= D << shift (Section 4.2 uses nextPow2(D) - 1, i.e.
// shift 0, with nextPow2 read as the next power of two strictly above D); the secondary
// modulus is p2 = 2 p1 + 1.  Keys are labels, values float32 weight sums.
//
// hashtableMaxKey is folded into the accumulation: every add returns the key's new sum,
// each lane keeps the maximum of (sum bits << 32 | ~label) over the adds it made, and the
// maxima are reduced over the lanes of the vertex.  A key's final sum is returned to the
// lane that made its last add and no observed sum exceeds a final sum (weights are >= 0),
// so the reduction equals the maximum over the table: the largest weight and, among equal
// weights, the smallest label (Section 4 item 5).
#include <mutex>

#include "sweep_kernels.cuh"

namespace lpa {

// The remainder multipliers are copied to each device once (every handle creation asks).
cudaError_t sweep_init_constants()
{
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    cudaError_t e = init_magic();
    if (e == cudaSuccess) e = sweep_init_constants_alt();
    if (e == cudaSuccess) e = sweep_init_constants_f64();
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

size_t max_dynamic_smem()
{
    query_device();
    return g_max_smem;
}

int num_sms()
{
    query_device();
    return g_num_sms;
}

__global__ void k_hub_begin(HArgs k)
{
    if (*k.active == 0) return;
    const WorkItem item = k.items[blockIdx.x];
    const SweepView a = view_of(k.gd, item.g);
    if (a.done) return;
    const HubArgs &h = k.gd[item.g].hub;
    for (int64_t t = item.start + threadIdx.x; t < item.start + item.count; t += blockDim.x) {
        const int32_t v = h.hub_v[t];
        uint8_t act = 1;                              // pull sweep: every hub is a candidate
        if (!a.pull) {
            act = a.flag_cur[v] != 0;
            if (act) a.flag_cur[v] = 0;               // mark processed
        }
        h.hub_act[t] = act;
        h.hub_seen[t] = 0;
        h.hub_best[t] = 0ull;
        h.hub_used[t] = 0u;
    }
}

// Clears the table slots a hub used in this sweep: slot by slot from the used list when
// few were used, or the whole table with coalesced stores when more than an eighth were.
template <int TPB>
__global__ void __launch_bounds__(TPB) k_hub_clear(HArgs k)
{
    if (*k.active == 0) return;
    const WorkItem item = k.items[blockIdx.x];
    const SweepView a = view_of(k.gd, item.g);
    if (a.done) return;
    const HubArgs &h = k.gd[item.g].hub;
    const int hh = h.slice_h[item.start];
    if (!h.hub_act[hh]) return;
    const bool packed = k.gd[item.g].int_weights != 0;
    const int64_t lo = (int64_t)h.slice_j[item.start] * kHubSlice;
    const int64_t cnt = h.hub_used[hh];
    const int64_t p1 = (int64_t)h.hub_p1[hh] + 1;   // the table's 2^b slots
    int32_t *Hk = h.tab_k + h.hub_tab[hh];
    float *Hv = h.tab_v + h.hub_tab[hh];
    double *Hd = h.tab_vd ? h.tab_vd + h.hub_tab[hh] : nullptr;
    unsigned long long *H = (unsigned long long *)h.tab_k + h.hub_tab[hh];
    auto clear = [&](int64_t q) {
        if (packed) {
            H[q] = kEmptySlot;
        } else {
            Hk[q] = kEmpty;
            if (Hd) Hd[q] = 0.0;
            else Hv[q] = 0.0f;
        }
    };
    if (cnt * 8 > p1) {
        if (lo >= p1) return;
        const int64_t hi = lo + kHubSlice < p1 ? lo + kHubSlice : p1;
        for (int64_t q = lo + threadIdx.x; q < hi; q += TPB) clear(q);
        return;
    }
    if (lo >= cnt) return;
    const int64_t hi = lo + kHubSlice < cnt ? lo + kHubSlice : cnt;
    const int32_t *ulist = h.used_list + h.used_base[hh];
    for (int64_t q = lo + threadIdx.x; q < hi; q += TPB) clear(ulist[q]);    // leave the table clear
}

__global__ void k_hub_move(HArgs k)
{
    if (*k.active == 0) return;
    const WorkItem item = k.items[blockIdx.x];
    const SweepView a = view_of(k.gd, item.g);
    if (a.done) return;
    const HubArgs &h = k.gd[item.g].hub;
    unsigned long long n_act = 0, n_edges = 0, n_moved = 0, n_marks = 0;
    for (int64_t hh = item.start + threadIdx.x; hh < item.start + item.count; hh += blockDim.x) {
        if (!h.hub_act[hh]) continue;
        if (a.pull && !h.hub_seen[hh]) continue;      // no neighbour moved: not active
        const int32_t v = h.hub_v[hh];
        const int32_t cur = (int32_t)((uint32_t)a.C[v] & kLabelMask);
        int32_t cstar = -1;
        bool moved;
        if (h.chunk_bv) {                             // float64 values: reduce the chunks' pairs
            BestD best;
            best_init(best);
            for (int32_t c = h.hub_c0[hh]; c < h.hub_c0[hh + 1]; ++c) best_merge(best, BestD{h.chunk_bv[c], h.chunk_bk[c]});
            moved = decide(best, cur, a.pl, cstar);
        } else {
            moved = decide(h.hub_best[hh], cur, a.pl, cstar);
        }
        const unsigned long long D = (unsigned long long)(a.off[v + 1] - a.off[v]);
        n_act += 1;
        n_edges += D;
        if (moved) {
            if (a.async_mode) {
                a.C[v] = cstar;
                __threadfence();
            } else {
                const unsigned long long pos = atomicAdd(a.mover_count, 1ull);
                a.mover_v[pos] = v;
                a.mover_c[pos] = cstar;
            }
            h.hub_act[hh] = a.mark ? 2 : 3;          // 2: k_hub_mark marks its neighbours now; 3: maybe after k_decide
            n_moved += 1;
            n_marks += D;
        }
    }
    unsigned long long *c = a.ctr + LPA_K_HUB_ACC * kCtrFields;
    if (n_act) atomicAdd(c + CTR_ACTIVE, n_act);
    if (n_edges) atomicAdd(c + CTR_EDGES, n_edges);
    if (n_moved) atomicAdd(c + CTR_MOVED, n_moved);
    if (n_marks) atomicAdd(c + CTR_MARKS, n_marks);
}

// Marks the neighbours of the moved hubs, a block per chunk of their rows: in the sweep
// (deferred = 0: hubs that moved in a marking sweep, into the next sweep's flags), or after
// k_decide (deferred = 1: hubs that moved in a sweep without marks when k_decide chose marks
// for the next sweep (rs->fin), into the flags of sweep rs->l, also after the run's last sweep).
template <int TPB>
__global__ void __launch_bounds__(TPB) k_hub_mark(HArgs k, int deferred)
{
    const WorkItem item = k.items[blockIdx.x];
    const GraphDev &G = k.gd[item.g];
    const HubArgs &h = G.hub;
    const int64_t c = item.start;
    uint8_t *flags;
    if (deferred) {
        const RunState *rs = G.rs;
        if (!rs->fin || h.hub_act[h.chunk_h[c]] != 3) return;
        flags = (rs->l & 1) ? G.flags1 : G.flags0;
    } else {
        if (*k.active == 0) return;
        const SweepView a = view_of(k.gd, item.g);
        if (a.done || h.hub_act[h.chunk_h[c]] != 2) return;
        flags = a.flag_next;
    }
    const int64_t e0 = h.chunk_e0[c], e1 = h.chunk_e1[c];
    mark_range(flags, G.idx, e0, e1, threadIdx.x, TPB);
}

// Synchronous mode, after a pull sweep: clear the moved bits of the previous sweep's movers
// (blockIdx.y: graph, blockIdx.x: stride over the list).  Runs before k_apply, which may set
// the bit again on a vertex that moved in both sweeps.
__global__ void k_apply_unmark(HArgs k)
{
    if (*k.active == 0) return;
    const WorkItem item = k.items[blockIdx.y];
    const SweepView a = view_of(k.gd, item.g);
    if (a.done || a.async_mode || !a.pull) return;
    const GraphDev &G = k.gd[item.g];
    const int l = G.rs->l;
    const int32_t *prev = ((l - 1) & 1) ? G.mover_v1 : G.mover_v;
    const unsigned long long n = G.mover_count[(l - 1) & 1];
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t v = prev[i];
        a.C[v] = (int32_t)((uint32_t)a.C[v] & kLabelMask);
    }
}

// Synchronous mode: publish the labels recorded during the sweep (blockIdx.y: graph,
// blockIdx.x: stride over its movers), with the moved bit when this sweep wrote no marks.
__global__ void k_apply(HArgs k)
{
    if (*k.active == 0) return;
    const WorkItem item = k.items[blockIdx.y];
    const SweepView a = view_of(k.gd, item.g);
    if (a.done || a.async_mode) return;
    const unsigned long long n = *a.mover_count;
    const uint32_t bit = a.mark ? 0u : kMovedBit;
    const GraphDev &G = k.gd[item.g];
    const RunState *rs = G.rs;
    const bool cc = rs->cc_period > 0 && rs->l % rs->cc_period == 0;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t v = a.mover_v[i];
        if (cc) {                                      // the Cross-Check needs the label before the sweep
            G.cc_prev[v] = a.C[v];
            G.cc_midx[v] = (int32_t)i;
        }
        a.C[v] = (int32_t)((uint32_t)a.mover_c[i] | bit);
    }
}

// ---------------------------------------------------------------------------------
// Cross-Check (Section 4.1) after a synchronous sweep l with l mod cc_period = 0.  The reading
// checks the movers in increasing id order: the move of x to p = C[x] is good iff vertex p
// holds label p at that moment.  For p = x, for p > x (not checked yet) and for p not a mover
// that is read directly from the labels after the sweep.  For a mover p < x it is K(p), where
// K(y) = [final label of y == y]; since y moved, K(y) = good(y) ? [p_y == y] : [prev_y == y],
// and for a dependent y (p_y < y, so p_y != y) that is [prev_y == y] AND NOT good(y).  So each
// dependent mover's K is a constant or the negation of its parent's K: a forest over smaller
// ids, resolved by pointer jumping.  Word of position j: negative = resolved, K in bit 0;
// otherwise parent position << 1 | parity (K_j = parity XOR K_parent).  Any snapshot of a
// parent's word keeps that relation, so the passes update in place.
__device__ __forceinline__ bool cc_sweep(const GraphDev &G)
{
    const RunState *rs = G.rs;
    return !rs->done && !rs->async_mode && rs->cc_period > 0 && rs->l % rs->cc_period == 0;
}

constexpr long long kCcResolved = (long long)0x8000000000000000ull;

__global__ void k_cc_init(HArgs k, unsigned *ctr)
{
    if (*k.active == 0) return;
    const GraphDev &G = k.gd[k.items[blockIdx.y].g];
    if (!cc_sweep(G)) return;
    const int l = G.rs->l;
    const int32_t *mv = (l & 1) ? G.mover_v1 : G.mover_v;
    const unsigned long long n = G.mover_count[l & 1];
    unsigned pending = 0;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t x = mv[j];
        const int32_t p = (int32_t)((uint32_t)G.C[x] & kLabelMask);
        const int32_t prev = G.cc_prev[x];
        const int32_t q = (p < x) ? G.cc_midx[p] : -1;
        long long word;
        if (p == x) {                                  // joined its own id: good, K = 1
            G.cc_par0[j] = -1;
            word = kCcResolved | 1;
        } else if (q >= 0) {                           // depends on the earlier mover p
            G.cc_par0[j] = q;
            if (prev == x) {
                word = ((long long)q << 1) | 1;        // K = NOT K(p)
                ++pending;
            } else {
                word = kCcResolved;                    // K = 0 whatever good is
            }
        } else {                                       // p not yet checked, or not a mover
            const bool good = (int32_t)((uint32_t)G.C[p] & kLabelMask) == p;
            G.cc_par0[j] = good ? -1 : -2;
            word = kCcResolved | (good ? 0 : (prev == x ? 1 : 0));
        }
        G.cc_word[j] = word;
    }
    if (pending) atomicAdd(ctr, pending);
}

// One pointer-jumping pass; skipped once a pass left nothing pending.
__global__ void k_cc_jump(HArgs k, unsigned *ctr, int pass)
{
    if (*k.active == 0 || ctr[pass] == 0) return;     // ctr[pass]: pending before this pass
    const GraphDev &G = k.gd[k.items[blockIdx.y].g];
    if (!cc_sweep(G)) return;
    const int l = G.rs->l;
    const unsigned long long n = G.mover_count[l & 1];
    unsigned pending = 0;
    volatile long long *W = G.cc_word;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const long long w = W[j];
        if (w < 0) continue;
        const long long wq = W[w >> 1];
        long long nw;
        if (wq < 0) {
            nw = kCcResolved | ((w ^ wq) & 1);
        } else {
            nw = (wq & ~1ll) | ((w ^ wq) & 1);
            ++pending;
        }
        W[j] = nw;
    }
    if (pending) atomicAdd(ctr + pass + 1, pending);
}

// Reverts the bad moves (back to the label before the sweep) and takes them off this sweep's
// move count (the apply slot's moved counter holds minus the reverted moves); clears the
// vertex -> position map.
__global__ void k_cc_revert(HArgs k, const unsigned *ctr)
{
    if (*k.active == 0) return;
    const GraphDev &G = k.gd[k.items[blockIdx.y].g];
    if (!cc_sweep(G)) return;
    const SweepView a = view_of(k.gd, k.items[blockIdx.y].g);
    const int l = G.rs->l;
    const int32_t *mv = (l & 1) ? G.mover_v1 : G.mover_v;
    const unsigned long long n = G.mover_count[l & 1];
    const bool resolved = ctr[kCcPasses] == 0;
    if (!resolved && blockIdx.x == 0 && threadIdx.x == 0) G.rs->cc_unresolved = 1;
    unsigned long long reverted = 0;
    for (unsigned long long j = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; j < n;
         j += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t x = mv[j];
        const int32_t q = G.cc_par0[j];
        const bool good = q >= 0 ? (G.cc_word[q] & 1) != 0 : q == -1;
        if (resolved && !good) {
            G.C[x] = G.cc_prev[x];
            ++reverted;
        }
        G.cc_midx[x] = -1;
    }
    if (reverted) atomicAdd(a.ctr + LPA_K_APPLY * kCtrFields + CTR_MOVED, (unsigned long long)(0 - reverted));
}


// After each sweep, per graph: the stop test of Algorithm 1 (after a sweep without Pick-Less,
// stop when dN / n < tolerance; stop at max_iters), then advance to the next sweep.
// Synchronous mode: the next sweep finds its active vertices (those with a neighbour that
// moved) from marks or from moved bits.  Marks cost a scattered byte store per entry of every
// mover; moved bits cost the next sweep a scan of every row.  So a sweep whose movers hold
// fewer than 1 / kFewMovedEntries of the CSR entries has its movers' neighbours marked: by the
// sweep itself when it was told to mark (rs->mark), else after it (rs->fin: k_finalize, and
// k_hub_mark for hubs); otherwise the next sweep pulls.  A sweep marks as it goes when the
// sweep before it moved few entries (a fresh run's first sweep moves most vertices and never
// does).  Cross-Check runs always mark.  Batches and the server (rs->adaptive = 0) keep one
// kernel variant per recorded sweep: only a fresh run's sweep 1 pulls and every later sweep
// marks as it goes (both variants in every sweep cost a batch of 4,096 graphs 5 %).
constexpr long long kFewMovedEntries = 4;

__global__ void k_decide(const GraphDev *gd, int n_graphs, int32_t *active)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_graphs) return;
    RunState *rs = gd[g].rs;
    if (rs->done) {
        rs->fin = 0;                                  // k_finalize has run once for this graph
        return;
    }
    const SweepView a = view_of(gd, g);
    long long dn = 0;
    for (int q = 0; q < LPA_NUM_KERNELS; ++q) dn += (long long)a.ctr[q * kCtrFields + CTR_MOVED];
    const int l = rs->l;
    int done = 0, conv = 0;
    if (!a.pl && (double)dn / (double)rs->n < rs->tol) {
        done = 1;
        conv = 1;
    } else if (l + 1 >= rs->max_iters) {
        done = 1;
    }
    if (!rs->async_mode) {
        long long me = 0;                             // CSR entries of this sweep's movers
        for (int q = 0; q < LPA_NUM_KERNELS; ++q) me += (long long)a.ctr[q * kCtrFields + CTR_MARKS];
        const long long m = (long long)gd[g].off[rs->n];
        const bool few = rs->cc_period > 0 || me * kFewMovedEntries < m;
        if (done) {
            rs->fin = rs->mark ? 0 : 1;               // this sweep's moved bits still stand
        } else if (!rs->adaptive) {
            rs->fin = 0;
            rs->pull = rs->mark ? 0 : 1;
            rs->mark = 1;
        } else {
            rs->fin = (!rs->mark && few) ? 1 : 0;     // mark after the sweep
            rs->pull = (rs->mark || few) ? 0 : 1;
            rs->mark = few ? 1 : 0;
        }
    }
    rs->l = l + 1;
    rs->last_dn = dn;
    rs->done = done;
    rs->converged = conv;
    gd[g].mover_count[(l + 1) & 1] = 0ull;           // the next sweep's list; this one stays for k_apply_unmark
    if (!done) atomicAdd(active, 1);
}

// After a synchronous sweep that set moved bits, when k_decide chose marks for the next sweep
// (rs->fin: few moved entries, or the run's last sweep, so that the saved state is that of a
// marking sweep): turn the bits into marks on the processed flags of sweep rs->l and clear
// them.  blockIdx.y: graph.  A warp takes 32 movers at a time: a lane marks the row of its
// own mover when it is short, and the warp marks the longer rows one after the other, all
// lanes on one row; hubs' rows are left to the chunked k_hub_mark.
constexpr int kFinalizeThreads = 256;
constexpr int64_t kFinalizeShort = kMarkUnroll;        // rows a lane marks alone
__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(const GraphDev *gd)
{
    const GraphDev &G = gd[blockIdx.y];
    const RunState *rs = G.rs;
    if (!rs->fin) return;
    const int last = rs->l - 1;
    const int32_t *mv = (last & 1) ? G.mover_v1 : G.mover_v;
    const unsigned long long n = G.mover_count[last & 1];
    uint8_t *flags = (rs->l & 1) ? G.flags1 : G.flags0;      // processed flags of sweep rs->l
    // in registers: the byte stores to the flags could otherwise alias the descriptor
    const int64_t *off = G.off;
    const int32_t *idx = G.idx;
    int32_t *C = G.C;
    const int64_t hub_deg = G.hub_deg;
    const int lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (kFinalizeThreads / 32);
    for (unsigned long long base = (blockIdx.x * (unsigned long long)(kFinalizeThreads / 32) + (threadIdx.x >> 5)) * 32;
         base < n; base += warps * 32) {
        int64_t e0 = 0, D = 0;
        if (base + lane < n) {
            const int32_t v = mv[base + lane];
            C[v] = (int32_t)((uint32_t)C[v] & kLabelMask);
            e0 = off[v];
            D = off[v + 1] - e0;
            if (D > hub_deg) D = 0;                   // a hub
        }
        if (D <= kFinalizeShort) mark_range(flags, idx, e0, e0 + D, 0, 1);
        unsigned longm = __ballot_sync(0xFFFFFFFFu, D > kFinalizeShort);
        while (longm) {
            const int src = __ffs(longm) - 1;
            longm &= longm - 1;
            const int64_t r0 = __shfl_sync(0xFFFFFFFFu, e0, src);
            const int64_t r1 = r0 + __shfl_sync(0xFFFFFFFFu, D, src);
            mark_range(flags, idx, r0, r1, lane, 32);
        }
    }
}

// Initial clear of all hub tables of a graph: `n` slots in the packed or the split layout.
__global__ void k_table_clear(int32_t *k, float *v, double *vd, int64_t n, int packed)
{
    unsigned long long *h = (unsigned long long *)k;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (packed) {
            h[i] = kEmptySlot;
        } else {
            k[i] = kEmpty;
            if (vd) vd[i] = 0.0;
            else v[i] = 0.0f;
        }
    }
}

template <int CS>
static int active_clusters()
{
    if (cudaFuncSetAttribute(k_hub_dsm<CS, false, kProbeQuadDoublePow2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDsmSmem) !=
            cudaSuccess ||
        (CS > 8 && cudaFuncSetAttribute(k_hub_dsm<CS, false, kProbeQuadDoublePow2>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                       cudaSuccess)) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS * 8, 1, 1);
    cfg.blockDim = dim3(kDsmThreads, 1, 1);
    cfg.dynamicSmemBytes = kDsmSmem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = CS;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_hub_dsm<CS, false, kProbeQuadDoublePow2>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int dsm_max_class_bits()
{
    static int cached = -1;                            // per process (one device type)
    if (cached >= 0) return cached;
    int bits = 0;
    if (active_clusters<2>() > 0) bits = 1;
    if (bits == 1 && active_clusters<4>() > 0) bits = 2;
    if (bits == 2 && active_clusters<8>() > 0) bits = 3;
    if (bits == 3 && active_clusters<16>() > 0) bits = 4;
    cached = bits;
    return bits;
}

cudaError_t enqueue_sweep(const SweepPlan &p, cudaStream_t s, LaunchHook *hook, int *launches)
{
    cudaError_t e = cudaMemsetAsync(p.queues, 0, sizeof(unsigned) * kQueueCount, s);
    if (e != cudaSuccess) return e;
    auto timed = [&](int slot, auto &&fn) -> cudaError_t {
        if (hook) hook->before(slot);
        cudaError_t r = fn();
        if (hook) hook->after(slot);
        if (launches) ++*launches;
        return r;
    };
    e = p.f64 ? launch_vertex_phase_f64(p, s, hook, launches)
              : (p.probe == kProbeQuadDoublePow2 ? launch_vertex_phase<kProbeQuadDoublePow2>(p, s, hook, launches)
                                                 : launch_vertex_phase_alt(p, s, hook, launches));
    if (e != cudaSuccess) return e;
    HArgs h{};
    h.gd = p.gd;
    h.active = p.active_count;
    h.chunk = p.hub_chunk;
    if (p.n_hub_items[HL_HUBS] > 0) {
        h.items = p.hub_items[HL_HUBS];
        e = timed(LPA_K_HUB_BEGIN, [&] {
            k_hub_begin<<<p.n_hub_items[HL_HUBS], 256, 0, s>>>(h);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
        e = p.f64 ? launch_hub_acc_phase_f64(p, h, s, hook, launches)
                  : (p.probe == kProbeQuadDoublePow2 ? launch_hub_acc_phase<kProbeQuadDoublePow2>(p, h, s, hook, launches)
                                                     : launch_hub_acc_phase_alt(p, h, s, hook, launches));
        if (e != cudaSuccess) return e;
        if (p.n_hub_items[HL_SLICES] > 0) {
            h.items = p.hub_items[HL_SLICES];
            e = timed(LPA_K_HUB_CLEAR, [&] {
                k_hub_clear<256><<<p.n_hub_items[HL_SLICES], 256, 0, s>>>(h);
                return cudaGetLastError();
            });
            if (e != cudaSuccess) return e;
        }
        h.items = p.hub_items[HL_HUBS];
        e = timed(LPA_K_HUB_MOVE, [&] {
            k_hub_move<<<p.n_hub_items[HL_HUBS], 128, 0, s>>>(h);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
        h.items = p.hub_items[HL_MARK];
        e = timed(LPA_K_HUB_MARK, [&] {
            k_hub_mark<512><<<p.n_hub_items[HL_MARK], 512, 0, s>>>(h, 0);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
    }
    h.items = p.per_graph;
    const unsigned bx = p.n_graphs == 1 ? (unsigned)(num_sms() * 4) : 8u;
    e = timed(LPA_K_APPLY, [&] {
        k_apply_unmark<<<dim3(bx, (unsigned)p.n_graphs), 256, 0, s>>>(h);
        k_apply<<<dim3(bx, (unsigned)p.n_graphs), 256, 0, s>>>(h);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;                         // k_apply_unmark
    if (p.cc_any) {                                    // Cross-Check of the graphs that ask for it
        e = cudaMemsetAsync(p.cc_ctr, 0, sizeof(unsigned) * (kCcPasses + 1), s);
        if (e != cudaSuccess) return e;
        k_cc_init<<<dim3(bx, (unsigned)p.n_graphs), 256, 0, s>>>(h, p.cc_ctr);
        for (int pass = 0; pass < kCcPasses; ++pass)
            k_cc_jump<<<dim3(bx, (unsigned)p.n_graphs), 256, 0, s>>>(h, p.cc_ctr, pass);
        k_cc_revert<<<dim3(bx, (unsigned)p.n_graphs), 256, 0, s>>>(h, p.cc_ctr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (launches) *launches += kCcPasses + 2;
    }
    e = cudaMemsetAsync(p.active_count, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    k_decide<<<(p.n_graphs + 127) / 128, 128, 0, s>>>(p.gd, p.n_graphs, p.active_count);
    k_finalize<<<dim3(bx, (unsigned)p.n_graphs), kFinalizeThreads, 0, s>>>(p.gd);
    if (launches) *launches += 2;
    if (p.n_hub_items[HL_MARK] > 0) {                 // the hubs' share of k_finalize's marks
        h.items = p.hub_items[HL_MARK];
        k_hub_mark<512><<<p.n_hub_items[HL_MARK], 512, 0, s>>>(h, 1);
        if (launches) ++*launches;
    }
    return cudaGetLastError();
}

cudaError_t launch_hub_table_clear(int32_t *k, float *v, int64_t slots, bool packed, cudaStream_t s, double *vd)
{
    if (slots <= 0) return cudaSuccess;
    query_device();
    int64_t blocks = (slots + 255) / 256;
    const int64_t cap = (int64_t)g_num_sms * 16;
    if (blocks > cap) blocks = cap;
    k_table_clear<<<(unsigned)blocks, 256, 0, s>>>(k, v, vd, slots, packed ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace lpa
