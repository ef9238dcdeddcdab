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
#include <cuda_runtime.h>
#include <stdint.h>

#include "lpa_internal.h"

namespace lpa {

// Multipliers for remainders by Mersenne numbers: c_magic[b] = ceil(2^64 / (2^b - 1))
// (0 for b = 1, where every remainder is 0).  a mod d = mulhi64(M * a, d) for 32-bit a
// and d (Lemire, Kaser and Kurz, "Faster remainder by direct computation", 2019).
__constant__ unsigned long long c_magic[33];

cudaError_t sweep_init_constants()
{
    unsigned long long h[33];
    h[0] = 0;
    for (int b = 1; b <= 32; ++b) {
        unsigned long long p = (b == 32) ? 0xFFFFFFFFull : ((1ull << b) - 1);
        h[b] = (p == 1) ? 0ull : (0xFFFFFFFFFFFFFFFFull / p + 1);
    }
    return cudaMemcpyToSymbol(c_magic, h, sizeof(h));
}

__device__ __forceinline__ uint32_t mod_mersenne(uint32_t a, uint32_t b, uint32_t p)
{
    unsigned long long low = c_magic[b] * (unsigned long long)a;
    return (uint32_t)__umul64hi(low, (unsigned long long)p);
}

// Label-weight values are float32, or uint32 when every weight is an integer and every
// weighted degree is below 2^24 (then each float32 sum is exact and equals the integer sum,
// and both compare the same way).  vbits gives bits that order like the value (values >= 0).
__device__ __forceinline__ uint32_t vbits(float w) { return __float_as_uint(w); }
__device__ __forceinline__ uint32_t vbits(uint32_t w) { return w; }
template <typename V> __device__ __forceinline__ V to_value(float w);
template <> __device__ __forceinline__ float to_value<float>(float w) { return w; }
template <> __device__ __forceinline__ uint32_t to_value<uint32_t>(float w) { return (uint32_t)w; }

template <typename V>
__device__ __forceinline__ unsigned long long pack_kv(V w, int32_t k)
{
    return ((unsigned long long)vbits(w) << 32) | (unsigned long long)(~(uint32_t)k);
}

__device__ __forceinline__ int32_t unpack_key(unsigned long long p)
{
    return (int32_t)(~(uint32_t)(p & 0xFFFFFFFFull));
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b)
{
    return a > b ? a : b;
}

// capacity 2^b - 1 >= x (x >= 1)
__device__ __forceinline__ uint32_t cap_bits(uint32_t x) { return 32u - __clz(x); }
__device__ __forceinline__ uint32_t cap_of_bits(uint32_t b) { return b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u); }

// One slot attempt of Algorithm 2: take slot s if it is empty or already holds k, add v
// and fold the new sum into `best`.  With TRACK a slot taken from empty is appended to the
// table's used list.
template <bool SHARED, bool TRACK, typename V>
__device__ __forceinline__ bool try_slot(int32_t *Hk, V *Hv, size_t s, int32_t k, V v,
                                         unsigned long long &best, uint32_t *ucnt, int32_t *ulist)
{
    if (!SHARED) {                                    // single owner: plain accesses
        const int32_t kk = Hk[s];
        if (kk == k || kk == kEmpty) {
            Hk[s] = k;
            const V nv = Hv[s] + v;
            Hv[s] = nv;
            best = umax64(best, pack_kv(nv, k));
            return true;
        }
        return false;
    }
    int32_t kk = *((volatile int32_t *)(Hk + s));
    if (kk == kEmpty) {
        const int32_t old = atomicCAS(Hk + s, kEmpty, k);
        if (old == kEmpty) {
            kk = k;
            if (TRACK) ulist[atomicAdd(ucnt, 1u)] = (int32_t)s;
        } else {
            kk = old;
        }
    }
    if (kk == k) {
        const V nv = atomicAdd(Hv + s, v) + v;
        best = umax64(best, pack_kv(nv, k));
        return true;
    }
    return false;
}

// hashtableAccumulate (Algorithm 2) with i and delta kept reduced mod p1 (same slots),
// then a linear scan from the last probed slot once the probe budget is spent.
template <bool SHARED, bool TRACK, typename V>
__device__ __forceinline__ void ht_accumulate(int32_t *Hk, V *Hv, int stride, uint32_t p1, uint32_t b,
                                              int32_t k, V v, unsigned long long &best, unsigned &fallbacks,
                                              uint32_t *ucnt = nullptr, int32_t *ulist = nullptr)
{
    const uint32_t uk = (uint32_t)k;
    uint32_t i = mod_mersenne(uk, b, p1);
    uint32_t delta = (p1 > 1u) ? 1u : 0u;
    uint32_t step = 0xFFFFFFFFu;                      // (k mod p2) mod p1, on first collision
    uint32_t s = i;
#pragma unroll 1
    for (int t = 0; t < kMaxRetries; ++t) {
        s = i;
        if (try_slot<SHARED, TRACK>(Hk, Hv, (size_t)s * stride, k, v, best, ucnt, ulist)) return;
        if (step == 0xFFFFFFFFu) {
            uint32_t q = mod_mersenne(uk, b + 1, 2u * p1 + 1u);
            if (q >= p1) q -= p1;
            if (q >= p1) q -= p1;
            step = q;
        }
        i += delta;
        if (i >= p1) i -= p1;
        unsigned long long d2 = 2ull * delta + step;    // < 3 p1
        if (d2 >= p1) d2 -= p1;
        if (d2 >= p1) d2 -= p1;
        delta = (uint32_t)d2;
    }
    ++fallbacks;
#pragma unroll 1
    for (uint32_t u = 1; u <= p1; ++u) {
        uint32_t q = s + u;
        if (q >= p1) q -= p1;
        if (try_slot<SHARED, TRACK>(Hk, Hv, (size_t)q * stride, k, v, best, ucnt, ulist)) return;
    }
}

template <int G>
__device__ __forceinline__ unsigned group_mask()
{
    if (G >= 32) return 0xFFFFFFFFu;
    const unsigned lane = threadIdx.x & 31u;
    return ((1u << (G & 31)) - 1u) << (lane & ~(unsigned)(G - 1));
}

template <int G>
__device__ __forceinline__ void group_sync()
{
    if (G > 1) __syncwarp(group_mask<G>());
}

template <int G>
__device__ __forceinline__ unsigned long long group_max(unsigned long long x)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x = umax64(x, __shfl_xor_sync(group_mask<G>(), x, o, G));
    return x;
}

// Lanes of one group (G lanes, aligned inside the warp) insert their (key, weight) pairs
// into the group's shared table.  Before the per-lane inserts, up to kPeel rounds take the
// key of the lowest pending lane, sum the weights of every lane holding that key with a
// shuffle reduction and insert the sum once: after a few sweeps most neighbours of a vertex
// share a handful of labels, and same-slot atomics would otherwise serialise.  Integer
// weights keep every partial sum exact, so the table contents do not depend on the order.
constexpr int kPeel = 3;

template <int G, bool SHARED, bool TRACK, typename V>
__device__ __forceinline__ void group_insert(int32_t *Hk, V *Hv, int stride, uint32_t p1, uint32_t b,
                                             bool has, int32_t k, V w, unsigned long long &best, unsigned &fb,
                                             uint32_t *ucnt = nullptr, int32_t *ulist = nullptr)
{
    if (G >= 2) {
        const unsigned gm = group_mask<G>();
        const int lane = threadIdx.x & 31;
        unsigned pend = __ballot_sync(gm, has);
#pragma unroll 1
        for (int r = 0; r < kPeel && pend; ++r) {
            const int leader = __ffs(pend) - 1;
            const int32_t kl = __shfl_sync(gm, k, leader);
            const bool mine = has && k == kl;
            const unsigned same = __ballot_sync(gm, mine);
            if (__popc(same) < 2) break;
            V sum = mine ? w : V(0);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(gm, sum, o);
            if (lane == leader) ht_accumulate<SHARED, TRACK>(Hk, Hv, stride, p1, b, kl, sum, best, fb, ucnt, ulist);
            if (mine) has = false;
            pend &= ~same;
        }
    }
    if (has) ht_accumulate<SHARED, TRACK>(Hk, Hv, stride, p1, b, k, w, best, fb, ucnt, ulist);
}

// hashtableClear of slots [0, p1] of a contiguous, 16-byte aligned table with 16-byte stores
// (p1 + 1 is a power of two, at least 4 slots are allocated).
// (Values are cleared to all-zero bits, which is 0 for both value types.)
__device__ __forceinline__ void clear_table_vec(int32_t *Hk, void *Hv, uint32_t p1, int first, int step)
{
    const uint32_t chunks = (p1 + 4u) >> 2;
    int4 *K4 = reinterpret_cast<int4 *>(Hk);
    int4 *V4 = reinterpret_cast<int4 *>(Hv);
    for (uint32_t q = first; q < chunks; q += step) {
        K4[q] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
        V4[q] = make_int4(0, 0, 0, 0);
    }
}

// The per-sweep view of one graph: what the sweep kernels read and write for an item of
// graph g, derived from its descriptor and run state.
struct SweepView {
    const int64_t *off;
    const int32_t *idx;
    const float *w;
    int32_t *C;
    uint8_t *flag_cur;         // unprocessed flags read (and cleared) by this sweep
    uint8_t *flag_next;        // flags set for the next sweep (== flag_cur in ASYNC mode)
    int32_t *mover_v, *mover_c;
    unsigned long long *mover_count;
    unsigned long long *ctr;   // this sweep's counters [LPA_NUM_KERNELS][kCtrFields]
    unsigned long long *fallbacks;
    const int32_t *lists;
    int32_t pl, async_mode, tshift, done;
};

__device__ __forceinline__ SweepView view_of(const GraphDev *gd, int g)
{
    const GraphDev &G = gd[g];
    const RunState *rs = G.rs;
    SweepView v;
    const int l = rs->l;
    v.done = rs->done;
    v.pl = (rs->pl_period > 0) && (l % rs->pl_period == 0);
    v.async_mode = rs->async_mode;
    v.off = G.off;
    v.idx = G.idx;
    v.w = G.w;
    v.C = G.C;
    if (v.async_mode) {
        v.flag_cur = G.flags0;
        v.flag_next = G.flags0;
    } else {
        v.flag_cur = (l & 1) ? G.flags1 : G.flags0;
        v.flag_next = (l & 1) ? G.flags0 : G.flags1;
    }
    v.mover_v = G.mover_v;
    v.mover_c = G.mover_c;
    v.mover_count = G.mover_count;
    const int slot = (l - rs->first) % (G.ctr_iters > 0 ? G.ctr_iters : 1);
    v.ctr = G.ctr + (size_t)(slot < 0 ? 0 : slot) * kPerSweep;
    v.fallbacks = G.fallbacks;
    v.lists = G.lists;
    v.tshift = G.tshift;
    return v;
}

// Warp-aggregated append of (v, c) to the synchronous mover list.  Every lane of the
// warp must call it.
__device__ __forceinline__ void append_movers(const SweepView &a, bool pred, int32_t v, int32_t c)
{
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, pred);
    if (!bal) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(bal) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(a.mover_count, (unsigned long long)__popc(bal));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    if (pred) {
        const unsigned long long pos = base + __popc(bal & ((1u << lane) - 1u));
        a.mover_v[pos] = v;
        a.mover_c[pos] = c;
    }
}

// Loads entry e of the row of v: (label of the neighbour, weight); has = false for e past
// the row end and for self-loops (Algorithm 1 skips j = i).
template <typename V>
__device__ __forceinline__ void load_entry(const SweepView &a, int32_t v, int64_t e, int64_t end, bool &has,
                                           int32_t &k, V &wv)
{
    has = e < end;
    k = 0;
    wv = V(0);
    if (has) {
        const int32_t j = a.idx[e];
        has = (j != v);
        if (has) {
            k = a.C[j];
            wv = a.w ? to_value<V>(a.w[e]) : V(1);
        }
    }
}

// Scans entries [start, end) of the row of v in rounds: each round covers U * step entries,
// lane offset `lane` inside each step.  All U entries of a round are loaded (index, weight,
// gathered label) before any of them is inserted, so U gathers per thread are in flight.
template <int G, bool SHARED, bool TRACK, int U, typename V>
__device__ __forceinline__ void scan_row(const SweepView &a, int32_t v, int64_t start, int64_t end, int step,
                                         int lane, int32_t *Hk, V *Hv, int stride, uint32_t p1, uint32_t b,
                                         unsigned long long &best, unsigned &fb, uint32_t *ucnt = nullptr,
                                         int32_t *ulist = nullptr, int round = 0)
{
    const int64_t adv = round ? round : (int64_t)step * U;   // a block-wide round for the CTA kernels
    for (int64_t eb = start; eb < end; eb += adv) {
        bool has[U];
        int32_t k[U];
        V wv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) load_entry(a, v, eb + (int64_t)u * step + lane, end, has[u], k[u], wv[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            group_insert<G, SHARED, TRACK>(Hk, Hv, stride, p1, b, has[u], k[u], wv[u], best, fb, ucnt, ulist);
    }
}

// Move rule of Algorithm 1: c* != C[i] and, on Pick-Less sweeps, c* < C[i].
__device__ __forceinline__ bool decide(unsigned long long best, int32_t cur, int pl, int32_t &cstar)
{
    if (best == 0) return false;                   // no neighbour label (isolated / self-loops only)
    cstar = unpack_key(best);
    return (cstar != cur) && (!pl || cstar < cur);
}

// ---------------------------------------------------------------------------------
// Kernel arguments common to the vertex kernels: the plan's graphs, this kernel's work items
// and work-queue counter, and the number of graphs still running (0: return at once).
struct KArgs {
    const GraphDev *gd;
    const WorkItem *items;
    int32_t n_items;
    int32_t slots;
    unsigned *queue;
    const int32_t *active;
    int32_t kslot;
    int32_t pad;
};

// Adds a warp's four counters and its fallback count to graph counters (every lane calls).
__device__ __forceinline__ void warp_flush(const SweepView &a, int kslot, unsigned act, unsigned edges,
                                           unsigned moved, unsigned marks, unsigned fb)
{
    act = __reduce_add_sync(0xFFFFFFFFu, act);
    edges = __reduce_add_sync(0xFFFFFFFFu, edges);
    moved = __reduce_add_sync(0xFFFFFFFFu, moved);
    marks = __reduce_add_sync(0xFFFFFFFFu, marks);
    fb = __reduce_add_sync(0xFFFFFFFFu, fb);
    if ((threadIdx.x & 31) == 0) {
        unsigned long long *c = a.ctr + kslot * kCtrFields;
        if (act) atomicAdd(c + CTR_ACTIVE, (unsigned long long)act);
        if (edges) atomicAdd(c + CTR_EDGES, (unsigned long long)edges);
        if (moved) atomicAdd(c + CTR_MOVED, (unsigned long long)moved);
        if (marks) atomicAdd(c + CTR_MARKS, (unsigned long long)marks);
        if (fb) atomicAdd(a.fallbacks, (unsigned long long)fb);
    }
}

// G lanes per vertex (G = 1: thread per vertex with a private table; G = 32: warp per
// vertex).  Persistent: each warp takes work items (a range of one graph's bucket list) from
// the queue and walks them 32/G vertices at a time.
template <int G, int TPB, typename V>
__global__ void __launch_bounds__(TPB) k_group(KArgs k)
{
    if (*k.active == 0) return;                        // every graph has stopped
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NG = TPB / G;
    constexpr int GPW = 32 / G;                        // groups per warp
    const int lane_w = threadIdx.x & 31;
    const int lane = (G == 1) ? 0 : (threadIdx.x & (G - 1));
    const int grp = threadIdx.x / G;
    const int gw = lane_w / G;                         // group within the warp
    int32_t *Hk;
    V *Hv;
    int stride;
    if (G == 1) {                      // interleaved: slot s of thread t at s * TPB + t
        Hk = (int32_t *)smem + threadIdx.x;
        Hv = (V *)(smem + (size_t)TPB * k.slots * sizeof(int32_t)) + threadIdx.x;
        stride = TPB;
    } else {
        Hk = (int32_t *)smem + (size_t)grp * k.slots;
        Hv = (V *)(smem + (size_t)NG * k.slots * sizeof(int32_t)) + (size_t)grp * k.slots;
        stride = 1;
    }
    for (;;) {
        int it = 0;
        if (lane_w == 0) it = (int)atomicAdd(k.queue, 1u);
        it = __shfl_sync(0xFFFFFFFFu, it, 0);
        if (it >= k.n_items) break;
        const WorkItem item = k.items[it];
        const SweepView a = view_of(k.gd, item.g);
        if (a.done) continue;
        unsigned fb = 0, c_act = 0, c_edges = 0, c_moved = 0, c_marks = 0;
        for (int64_t wb = 0; wb < item.count; wb += GPW) {          // uniform per warp
            const int64_t gi = wb + gw;
            int32_t v = -1;
            bool act = false;
            if (gi < item.count) {
                v = __ldg(a.lists + item.start + gi);
                if (lane == 0) {
                    act = a.flag_cur[v] != 0;
                    if (act) a.flag_cur[v] = 0;           // mark processed
                }
            }
            if (G > 1) act = __shfl_sync(group_mask<G>(), act, 0, G);
            int32_t cstar = -1;
            bool moved = false;
            if (act) {
                const int64_t o0 = a.off[v], o1 = a.off[v + 1];
                const uint32_t D = (uint32_t)(o1 - o0);
                const uint32_t b = cap_bits(D << a.tshift);    // capacity >= D << tshift
                const uint32_t p1 = cap_of_bits(b);
                if (G == 1) {
                    for (uint32_t s = 0; s < p1; ++s) {        // hashtableClear
                        Hk[(size_t)s * stride] = kEmpty;
                        Hv[(size_t)s * stride] = V(0);
                    }
                } else {
                    group_sync<G>();                           // previous vertex's inserts are done
                    clear_table_vec(Hk, Hv, p1, lane, G);
                    group_sync<G>();
                }
                const int32_t cur = a.C[v];
                unsigned long long best = 0;
                scan_row<G, (G > 1), false, 1>(a, v, o0, o1, G, lane, Hk, Hv, stride, p1, b, best, fb);
                best = group_max<G>(best);                     // hashtableMaxKey
                moved = decide(best, cur, a.pl, cstar);
                if (moved) {
                    if (a.async_mode && lane == 0) {
                        a.C[v] = cstar;
                        __threadfence();
                    }
                    group_sync<G>();
                    for (int64_t e = o0 + lane; e < o1; e += G) a.flag_next[a.idx[e]] = 1;   // mark neighbours
                }
                if (lane == 0) {
                    c_act += 1;
                    c_edges += D;
                    if (moved) {
                        c_moved += 1;
                        c_marks += D;
                    }
                }
            }
            if (!a.async_mode) append_movers(a, moved && lane == 0, v, cstar);
        }
        warp_flush(a, k.kslot, c_act, c_edges, c_moved, c_marks, fb);
    }
}

// One thread block per vertex; the table (up to k.slots entries) lives in dynamic smem.
// Persistent: each block takes work items from the queue and walks their vertices.
template <int TPB, typename V>
__global__ void __launch_bounds__(TPB) k_cta(KArgs k)
{
    if (*k.active == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t *Hk = (int32_t *)smem;
    V *Hv = (V *)(smem + (size_t)k.slots * sizeof(int32_t));
    __shared__ int s_item, s_act;
    __shared__ int32_t s_v;
    __shared__ unsigned long long s_best[TPB / 32];
    for (;;) {
        __syncthreads();                               // s_item and s_best of the last round are consumed
        if (threadIdx.x == 0) s_item = (int)atomicAdd(k.queue, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= k.n_items) break;
        const WorkItem item = k.items[it];
        const SweepView a = view_of(k.gd, item.g);
        if (a.done) continue;
        unsigned fb = 0;
        unsigned long long c_act = 0, c_edges = 0, c_moved = 0, c_marks = 0;
        for (int64_t gi = 0; gi < item.count; ++gi) {
            __syncthreads();                           // the previous vertex is finished
            if (threadIdx.x == 0) {
                const int32_t v0 = __ldg(a.lists + item.start + gi);
                const int act = a.flag_cur[v0] != 0;
                if (act) a.flag_cur[v0] = 0;           // mark processed
                s_act = act;
                s_v = v0;
            }
            __syncthreads();
            if (!s_act) continue;                      // uniform for the block
            const int32_t v = s_v;
            const int64_t o0 = a.off[v], o1 = a.off[v + 1];
            const uint32_t D = (uint32_t)(o1 - o0);
            const uint32_t b = cap_bits(D << a.tshift);
            const uint32_t p1 = cap_of_bits(b);
            clear_table_vec(Hk, Hv, p1, threadIdx.x, TPB);
            __syncthreads();
            const int32_t cur = a.C[v];
            unsigned long long best = 0;
            constexpr int U = TPB >= 1024 ? 2 : 1;         // loads in flight per thread
            scan_row<32, true, false, U>(a, v, o0 + (threadIdx.x & ~31) * U, o1, 32, threadIdx.x & 31, Hk, Hv, 1,
                                         p1, b, best, fb, nullptr, nullptr, TPB * U);
            best = group_max<32>(best);
            if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
            __syncthreads();
            best = 0;
#pragma unroll
            for (int w = 0; w < TPB / 32; ++w) best = umax64(best, s_best[w]);
            int32_t cstar = -1;
            const bool moved = decide(best, cur, a.pl, cstar);
            if (moved) {
                if (threadIdx.x == 0) {
                    if (a.async_mode) {
                        a.C[v] = cstar;
                        __threadfence();
                    } else {
                        const unsigned long long pos = atomicAdd(a.mover_count, 1ull);
                        a.mover_v[pos] = v;
                        a.mover_c[pos] = cstar;
                    }
                }
                if (a.async_mode) __syncthreads();
                for (int64_t e = o0 + threadIdx.x; e < o1; e += TPB) a.flag_next[a.idx[e]] = 1;
            }
            if (threadIdx.x == 0) {
                c_act += 1;
                c_edges += D;
                if (moved) {
                    c_moved += 1;
                    c_marks += D;
                }
            }
        }
        if (threadIdx.x == 0) {
            unsigned long long *c = a.ctr + k.kslot * kCtrFields;
            if (c_act) atomicAdd(c + CTR_ACTIVE, c_act);
            if (c_edges) atomicAdd(c + CTR_EDGES, c_edges);
            if (c_moved) atomicAdd(c + CTR_MOVED, c_moved);
            if (c_marks) atomicAdd(c + CTR_MARKS, c_marks);
        }
        if (fb) atomicAdd(a.fallbacks, (unsigned long long)fb);
    }
}

// ---------------------------------------------------------------------------------
// Hubs: tables in HBM shared by several blocks.  Per sweep: begin (take the processed
// flag), accumulate (a block per CSR chunk; each block folds its running maximum into
// hub_best), clear (a block per slice of the used-slot list or of the table), move (the
// decision), mark (a block per CSR chunk of the hubs that moved).  Items: begin and move take
// a graph's hubs [start, start + count); accumulate, clear and mark take one chunk / slice.
struct HArgs {
    const GraphDev *gd;
    const WorkItem *items;
    const int32_t *active;
    int32_t chunk;
    int32_t pad;
};

__global__ void k_hub_begin(HArgs k)
{
    if (*k.active == 0) return;
    const WorkItem item = k.items[blockIdx.x];
    const SweepView a = view_of(k.gd, item.g);
    if (a.done) return;
    const HubArgs &h = k.gd[item.g].hub;
    for (int64_t t = item.start + threadIdx.x; t < item.start + item.count; t += blockDim.x) {
        const int32_t v = h.hub_v[t];
        const uint8_t act = a.flag_cur[v] != 0;
        if (act) a.flag_cur[v] = 0;                   // mark processed
        h.hub_act[t] = act;
        h.hub_best[t] = 0ull;
        h.hub_used[t] = 0u;
    }
}

// Slots taken from empty are collected in a block-local list in shared memory and copied to
// the hub's used list with one global atomic per block.
template <int TPB, typename V>
__global__ void __launch_bounds__(TPB) k_hub_acc(HArgs k)
{
    if (*k.active == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t *s_list = (int32_t *)smem;                 // [chunk]
    __shared__ unsigned long long s_best[TPB / 32];
    __shared__ uint32_t s_cnt, s_base;
    const WorkItem item = k.items[blockIdx.x];
    const SweepView a = view_of(k.gd, item.g);
    if (a.done) return;
    const HubArgs &h = k.gd[item.g].hub;
    const int64_t c = item.start;
    const int hh = h.chunk_h[c];
    if (!h.hub_act[hh]) return;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int32_t v = h.hub_v[hh];
    const uint32_t p1 = h.hub_p1[hh], b = h.hub_b[hh];
    int32_t *Hk = h.tab_k + h.hub_tab[hh];
    V *Hv = reinterpret_cast<V *>(h.tab_v) + h.hub_tab[hh];
    const int64_t e0 = h.chunk_e0[c], e1 = h.chunk_e1[c];
    unsigned fb = 0;
    unsigned long long best = 0;
    scan_row<32, true, true, 2>(a, v, e0 + (threadIdx.x & ~31) * 2, e1, 32, threadIdx.x & 31, Hk, Hv, 1, p1, b,
                                best, fb, &s_cnt, s_list, TPB * 2);
    if (fb) atomicAdd(a.fallbacks, (unsigned long long)fb);
    best = group_max<32>(best);
    if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < TPB / 32; ++w) best = umax64(best, s_best[w]);
        if (best) atomicMax(h.hub_best + hh, best);
        s_base = s_cnt ? atomicAdd(h.hub_used + hh, s_cnt) : 0u;
    }
    __syncthreads();
    int32_t *ulist = h.used_list + h.used_base[hh] + s_base;
    for (uint32_t q = threadIdx.x; q < s_cnt; q += TPB) ulist[q] = s_list[q];
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
    const int64_t lo = (int64_t)h.slice_j[item.start] * kHubSlice;
    const int64_t cnt = h.hub_used[hh];
    const int64_t p1 = h.hub_p1[hh];
    int32_t *Hk = h.tab_k + h.hub_tab[hh];
    float *Hv = h.tab_v + h.hub_tab[hh];
    if (cnt * 8 > p1) {
        if (lo >= p1) return;
        const int64_t hi = lo + kHubSlice < p1 ? lo + kHubSlice : p1;
        for (int64_t q = lo + threadIdx.x; q < hi; q += TPB) {
            Hk[q] = kEmpty;
            Hv[q] = 0.0f;
        }
        return;
    }
    if (lo >= cnt) return;
    const int64_t hi = lo + kHubSlice < cnt ? lo + kHubSlice : cnt;
    const int32_t *ulist = h.used_list + h.used_base[hh];
    for (int64_t q = lo + threadIdx.x; q < hi; q += TPB) {
        const int32_t s = ulist[q];
        Hk[s] = kEmpty;                                // leave the table clear for the next sweep
        Hv[s] = 0.0f;
    }
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
        const int32_t v = h.hub_v[hh];
        const int32_t cur = a.C[v];
        int32_t cstar = -1;
        const bool moved = decide(h.hub_best[hh], cur, a.pl, cstar);
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
            h.hub_act[hh] = 2;
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

template <int TPB>
__global__ void __launch_bounds__(TPB) k_hub_mark(HArgs k)
{
    if (*k.active == 0) return;
    const WorkItem item = k.items[blockIdx.x];
    const SweepView a = view_of(k.gd, item.g);
    if (a.done) return;
    const HubArgs &h = k.gd[item.g].hub;
    const int64_t c = item.start;
    if (h.hub_act[h.chunk_h[c]] != 2) return;
    const int64_t e0 = h.chunk_e0[c], e1 = h.chunk_e1[c];
    for (int64_t e = e0 + threadIdx.x; e < e1; e += TPB) a.flag_next[a.idx[e]] = 1;
}

// Synchronous mode: publish the labels recorded during the sweep (blockIdx.y: graph,
// blockIdx.x: stride over its movers).
__global__ void k_apply(HArgs k)
{
    if (*k.active == 0) return;
    const WorkItem item = k.items[blockIdx.y];
    const SweepView a = view_of(k.gd, item.g);
    if (a.done || a.async_mode) return;
    const unsigned long long n = *a.mover_count;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        a.C[a.mover_v[i]] = a.mover_c[i];
}

// After each sweep, per graph: the stop test of Algorithm 1 (after a sweep without Pick-Less,
// stop when dN / n < tolerance; stop at max_iters), then advance to the next sweep.
__global__ void k_decide(const GraphDev *gd, int n_graphs, int32_t *active)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_graphs) return;
    RunState *rs = gd[g].rs;
    if (rs->done) return;
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
    rs->l = l + 1;
    rs->last_dn = dn;
    rs->done = done;
    rs->converged = conv;
    *gd[g].mover_count = 0ull;
    if (!done) atomicAdd(active, 1);
}

__global__ void k_table_clear(int32_t *k, float *v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        k[i] = kEmpty;
        v[i] = 0.0f;
    }
}

// ---------------------------------------------------------------------------------
// launchers

static int g_num_sms = 0;
static size_t g_max_smem = 0;

static void query_device()
{
    if (g_num_sms) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    int smem = 0;
    cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    g_max_smem = (size_t)smem;
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

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename K>
static int64_t persistent_grid(K kernel, int threads, size_t smem, int64_t work_blocks)
{
    query_device();
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t cap = (int64_t)g_num_sms * per_sm;
    return work_blocks < cap ? work_blocks : cap;
}

template <int G, int TPB, typename V>
static cudaError_t launch_gv(const KArgs &k, cudaStream_t s)
{
    constexpr int NG = TPB / G;
    const size_t smem = (size_t)NG * k.slots * (sizeof(int32_t) + sizeof(V));
    cudaError_t e = set_smem(k_group<G, TPB, V>, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = persistent_grid(k_group<G, TPB, V>, TPB, smem, ((int64_t)k.n_items + 7) / 8 * 8);
    k_group<G, TPB, V><<<(unsigned)(blocks < 1 ? 1 : blocks), TPB, smem, s>>>(k);
    return cudaGetLastError();
}

template <int G, int TPB>
static cudaError_t launch_g(const KArgs &k, bool int_w, cudaStream_t s)
{
    return int_w ? launch_gv<G, TPB, uint32_t>(k, s) : launch_gv<G, TPB, float>(k, s);
}

template <int TPB, typename V>
static cudaError_t launch_cv(const KArgs &k, cudaStream_t s)
{
    const size_t smem = (size_t)k.slots * (sizeof(int32_t) + sizeof(V));
    cudaError_t e = set_smem(k_cta<TPB, V>, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = persistent_grid(k_cta<TPB, V>, TPB, smem, k.n_items);
    k_cta<TPB, V><<<(unsigned)(blocks < 1 ? 1 : blocks), TPB, smem, s>>>(k);
    return cudaGetLastError();
}

static cudaError_t launch_cta(const KArgs &k, int threads, bool int_w, cudaStream_t s)
{
    switch (threads) {
    case 64: return int_w ? launch_cv<64, uint32_t>(k, s) : launch_cv<64, float>(k, s);
    case 128: return int_w ? launch_cv<128, uint32_t>(k, s) : launch_cv<128, float>(k, s);
    case 256: return int_w ? launch_cv<256, uint32_t>(k, s) : launch_cv<256, float>(k, s);
    case 512: return int_w ? launch_cv<512, uint32_t>(k, s) : launch_cv<512, float>(k, s);
    case 1024: return int_w ? launch_cv<1024, uint32_t>(k, s) : launch_cv<1024, float>(k, s);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t launch_vertex(const SweepPlan &p, int b, cudaStream_t s)
{
    KArgs k{};
    k.gd = p.gd;
    k.items = p.items[b];
    k.n_items = p.n_items[b];
    k.slots = p.slots[b];
    k.queue = p.queues + b;
    k.active = p.active_count;
    k.kslot = b;                                       // bucket index == kernel slot
    const bool iw = p.int_weights != 0;
    switch (b) {
    case B_THREAD: return launch_g<1, 128>(k, iw, s);
    case B_GROUP:
        switch (p.group_lanes) {
        case 2: return launch_g<2, 256>(k, iw, s);
        case 4: return launch_g<4, 256>(k, iw, s);
        case 8: return launch_g<8, 256>(k, iw, s);
        case 16: return launch_g<16, 256>(k, iw, s);
        default: return cudaErrorInvalidValue;
        }
    case B_WARP: return launch_g<32, 256>(k, iw, s);
    case B_CTA: return launch_cta(k, p.cta_threads, iw, s);
    case B_CTA_LARGE: return launch_cta(k, p.cta_large_threads, iw, s);
    case B_CTA_XL: return launch_cta(k, p.cta_xl_threads, iw, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t enqueue_sweep(const SweepPlan &p, cudaStream_t s, LaunchHook *hook, int *launches)
{
    cudaError_t e = cudaMemsetAsync(p.queues, 0, sizeof(unsigned) * B_COUNT, s);
    if (e != cudaSuccess) return e;
    auto timed = [&](int slot, auto &&fn) -> cudaError_t {
        if (hook) hook->before(slot);
        cudaError_t r = fn();
        if (hook) hook->after(slot);
        if (launches) ++*launches;
        return r;
    };
    for (int b = B_THREAD; b <= B_CTA_XL; ++b) {
        if (p.n_items[b] <= 0) continue;
        e = timed(b, [&] { return launch_vertex(p, b, s); });
        if (e != cudaSuccess) return e;
    }
    HArgs h{};
    h.gd = p.gd;
    h.active = p.active_count;
    h.chunk = p.hub_chunk;
    if (p.n_hub_hubs > 0) {
        h.items = p.hub_hubs;
        e = timed(LPA_K_HUB_BEGIN, [&] {
            k_hub_begin<<<p.n_hub_hubs, 256, 0, s>>>(h);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
        h.items = p.hub_chunks;
        e = timed(LPA_K_HUB_ACC, [&] {
            const size_t smem = (size_t)p.hub_chunk * sizeof(int32_t);
            if (p.int_weights) {
                cudaError_t r = set_smem(k_hub_acc<1024, uint32_t>, smem);
                if (r != cudaSuccess) return r;
                k_hub_acc<1024, uint32_t><<<p.n_hub_chunks, 1024, smem, s>>>(h);
            } else {
                cudaError_t r = set_smem(k_hub_acc<1024, float>, smem);
                if (r != cudaSuccess) return r;
                k_hub_acc<1024, float><<<p.n_hub_chunks, 1024, smem, s>>>(h);
            }
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
        h.items = p.hub_slices;
        e = timed(LPA_K_HUB_CLEAR, [&] {
            k_hub_clear<256><<<p.n_hub_slices, 256, 0, s>>>(h);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
        h.items = p.hub_hubs;
        e = timed(LPA_K_HUB_MOVE, [&] {
            k_hub_move<<<p.n_hub_hubs, 128, 0, s>>>(h);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
        h.items = p.hub_chunks;
        e = timed(LPA_K_HUB_MARK, [&] {
            k_hub_mark<512><<<p.n_hub_chunks, 512, 0, s>>>(h);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
    }
    h.items = p.per_graph;
    e = timed(LPA_K_APPLY, [&] {
        const unsigned bx = p.n_graphs == 1 ? (unsigned)(num_sms() * 4) : 8u;
        k_apply<<<dim3(bx, (unsigned)p.n_graphs), 256, 0, s>>>(h);
        return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p.active_count, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    k_decide<<<(p.n_graphs + 127) / 128, 128, 0, s>>>(p.gd, p.n_graphs, p.active_count);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_hub_table_clear(int32_t *k, float *v, int64_t slots, cudaStream_t s)
{
    if (slots <= 0) return cudaSuccess;
    query_device();
    int64_t blocks = (slots + 255) / 256;
    const int64_t cap = (int64_t)g_num_sms * 16;
    if (blocks > cap) blocks = cap;
    k_table_clear<<<(unsigned)blocks, 256, 0, s>>>(k, v, slots);
    return cudaGetLastError();
}

}  // namespace lpa
