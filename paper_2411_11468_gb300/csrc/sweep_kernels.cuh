// Table-dependent sweep kernels of liblpa.so and their launchers, shared by two translation
// units: lpa_sweep.cu instantiates them for Algorithm 2's quadratic-double probe fixed at
// compile time (the default path), lpa_sweep_alt.cu once more with the probe scheme read at
// run time (the probe-scheme comparison of Section 4.2).  Everything here has internal or
// template linkage.
//
// One label-propagation sweep (Algorithm 1, lpaMove) over the
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
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lpa_internal.h"

namespace cg = cooperative_groups;

namespace lpa {


// Multipliers for remainders by Mersenne numbers: c_magic[b] = ceil(2^64 / (2^b - 1))
// (0 for b = 1, where every remainder is 0).  a mod d = mulhi64(M * a, d) for 32-bit a
// and d (Lemire, Kaser and Kurz, "Faster remainder by direct computation", 2019).  One copy
// per translation unit that includes this header, filled by init_magic().
static __constant__ unsigned long long c_magic[33];

static cudaError_t init_magic()
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
template <> __device__ __forceinline__ double to_value<double>(float w) { return (double)w; }

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

// Running arg-max of a lane (largest sum, smallest label among equal sums).  uint32 and
// float32 sums: one 64-bit word, pack_kv(sum, label), whose unsigned maximum is the arg-max
// (0 = none).  float64 sums (lpa_tuning.float_values = 2) do not fit beside a label in 64
// bits: the pair itself (k < 0 = none).
struct BestD {
    double v;
    int32_t k;
};
template <typename V> struct BestOf {
    using type = unsigned long long;
};
template <> struct BestOf<double> {
    using type = BestD;
};

__device__ __forceinline__ void best_init(unsigned long long &b) { b = 0ull; }
__device__ __forceinline__ void best_init(BestD &b)
{
    b.v = -1.0;
    b.k = -1;
}
template <typename V>
__device__ __forceinline__ void best_add(unsigned long long &b, V w, int32_t k) { b = umax64(b, pack_kv(w, k)); }
__device__ __forceinline__ void best_add(BestD &b, double w, int32_t k)
{
    if (w > b.v || (w == b.v && k < b.k)) {
        b.v = w;
        b.k = k;
    }
}
__device__ __forceinline__ void best_merge(unsigned long long &b, unsigned long long o) { b = umax64(b, o); }
__device__ __forceinline__ void best_merge(BestD &b, const BestD &o)
{
    if (o.k >= 0) best_add(b, o.v, o.k);
}

// capacity 2^b - 1 >= x (x >= 1)
__device__ __forceinline__ uint32_t cap_bits(uint32_t x) { return 32u - __clz(x); }
__device__ __forceinline__ uint32_t cap_of_bits(uint32_t b) { return b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u); }

// Table layouts.  Split: keys and values in two arrays (slot s at index s * stride).  Packed
// (integer sums only): one 64-bit word per slot, key in the high half and the uint32 sum in
// the low half, so taking an empty slot is one compare-and-swap that also stores the first
// weight, and adding to a present key is one add (sums stay below 2^24, so the low half
// never carries into the key).  Both hold the same (key, sum) pairs at the same slots.
// Probe schemes of Section 4.2 (lpa_tuning.probe): the quadratic-double hybrid of Algorithm 2
// (the default), and for comparison linear probing, quadratic probing and double hashing.
// PROBE >= 0 fixes the scheme at compile time (the default kernels); PROBE = kProbeRuntime
// reads it from the table (the comparison kernels, in their own translation unit).
// kProbeQuadDoublePow2 keeps Algorithm 2's recurrence (i <- i + delta, delta <- 2 delta + h2(k))
// but takes it modulo the table's whole power-of-two allocation (2^b slots, mask p1 = 2^b - 1)
// with multiplicative first and second hashes: the first slot is the top b bits of k times an
// odd constant (Fibonacci hashing), the second hash is odd, so every step is odd.  It replaces
// the Mersenne remainders (k mod p1, k mod p2) by two multiplies and masks, and it disperses
// ids that share their low bits or have few bits set, as the unpermuted ids of R-MAT graphs do.
enum { kProbeRuntime = -1, kProbeQuadDouble = 0, kProbeLinear = 1, kProbeQuadratic = 2, kProbeDouble = 3,
       kProbeQuadDoublePow2 = 4 };
constexpr uint32_t kHashMul1 = 0x9E3779B1u;   // 2^32 / golden ratio, odd
constexpr uint32_t kHashMul2 = 0x85EBCA77u;   // odd multiplier of the second hash

template <typename V, int PROBE>
struct SplitTable {
    using Val = V;
    static constexpr int kProbe = PROBE;
    int32_t *k;
    V *v;
    int stride;
    int probe = kProbeQuadDouble;
};

// READ_FIRST: a slot is read before it is updated (HBM hub tables: after the first sweep most
// labels are present, and a read plus an add is cheaper than a compare-and-swap that fails on
// a contended line); otherwise (shared memory) the compare-and-swap comes first and the read
// is saved when the slot is empty.
template <int PROBE, bool READ_FIRST = false>
struct PackedTable {
    using Val = uint32_t;
    static constexpr int kProbe = PROBE;
    unsigned long long *h;
    int stride;
    int probe = kProbeQuadDouble;
};

constexpr unsigned long long kEmptySlot = 0xFFFFFFFF00000000ull;   // key -1, sum 0

// One slot attempt of Algorithm 2: take slot s if it is empty or already holds k, add v
// and fold the new sum into `best`.  With TRACK a slot taken from empty is appended to the
// table's used list.
template <bool SHARED, bool TRACK, typename V, int PROBE>
__device__ __forceinline__ bool try_slot(const SplitTable<V, PROBE> &T, size_t s, int32_t k, V v,
                                         typename BestOf<V>::type &best, uint32_t *ucnt, int32_t *ulist)
{
    int32_t *Hk = T.k;
    V *Hv = T.v;
    if (!SHARED) {                                    // single owner: plain accesses
        const int32_t kk = Hk[s];
        if (kk == k || kk == kEmpty) {
            Hk[s] = k;
            const V nv = Hv[s] + v;
            Hv[s] = nv;
            best_add(best, nv, k);
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
        best_add(best, nv, k);
        return true;
    }
    return false;
}

// Shared (atomic) update of one packed slot at p (slot index s for the used list).
template <bool TRACK, bool READ_FIRST>
__device__ __forceinline__ bool packed_update(unsigned long long *p, size_t s, int32_t k, uint32_t v,
                                              unsigned long long &best, uint32_t *ucnt, int32_t *ulist)
{
    const uint32_t uk = (uint32_t)k;
    uint32_t ck = READ_FIRST ? (uint32_t)(*((volatile unsigned long long *)p) >> 32) : 0xFFFFFFFFu;
    if (ck == 0xFFFFFFFFu) {
        const unsigned long long old = atomicCAS(p, kEmptySlot, ((unsigned long long)uk << 32) | v);
        if (old == kEmptySlot) {
            if (TRACK) ulist[atomicAdd(ucnt, 1u)] = (int32_t)s;
            best = umax64(best, pack_kv(v, k));
            return true;
        }
        ck = (uint32_t)(old >> 32);
    }
    if (ck == uk) {
        // 32-bit add on the sum half (the low word, at the lower address): native in shared
        // memory, unlike a 64-bit add.  The key half never changes once the slot is taken, so
        // a concurrent compare-and-swap on the slot fails on the key whatever the sum.
        const uint32_t nv = atomicAdd(reinterpret_cast<uint32_t *>(p), v) + v;
        best = umax64(best, pack_kv(nv, k));
        return true;
    }
    return false;
}

template <bool SHARED, bool TRACK, int PROBE, bool READ_FIRST>
__device__ __forceinline__ bool try_slot(const PackedTable<PROBE, READ_FIRST> &T, size_t s, int32_t k, uint32_t v,
                                         unsigned long long &best, uint32_t *ucnt, int32_t *ulist)
{
    unsigned long long *p = T.h + s;
    if (!SHARED) {
        const uint32_t uk = (uint32_t)k;
        const unsigned long long cur = *p;
        const uint32_t ck = (uint32_t)(cur >> 32);
        if (ck == uk || ck == 0xFFFFFFFFu) {
            const uint32_t nv = (uint32_t)cur + v;       // an empty slot holds sum 0
            *p = ((unsigned long long)uk << 32) | nv;
            best = umax64(best, pack_kv(nv, k));
            return true;
        }
        return false;
    }
    return packed_update<TRACK, READ_FIRST>(p, s, k, v, best, ucnt, ulist);
}

// A hub table spread over the shared memory of the blocks of a thread-block cluster (packed
// layout): slot s lives in block s >> lb at index s & (2^lb - 1) of that block's slice, and
// is reached through the cluster's distributed shared memory.
template <int PROBE>
struct ClusterTable {
    using Val = uint32_t;
    static constexpr int kProbe = PROBE;
    unsigned long long *base;  // this block's slice
    uint32_t lb;               // log2 of the slots per block
    int stride;                // 1
    int probe = kProbeQuadDouble;
};

template <bool SHARED, bool TRACK, int PROBE>
__device__ __forceinline__ bool try_slot(const ClusterTable<PROBE> &T, size_t s, int32_t k, uint32_t v,
                                         unsigned long long &best, uint32_t *ucnt, int32_t *ulist)
{
    unsigned long long *p = cg::this_cluster().map_shared_rank(T.base, (unsigned)(s >> T.lb)) +
                            (s & (((size_t)1 << T.lb) - 1));
    return packed_update<TRACK, true>(p, s, k, v, best, ucnt, ulist);
}

// hashtableAccumulate (Algorithm 2) with i and delta kept reduced mod p1 (same slots),
// then a linear scan from the last probed slot once the probe budget is spent.  The probe
// step follows the table's scheme: Algorithm 2's delta <- 2 delta + (k mod p2) from delta = 1;
// linear: delta = 1; quadratic: delta <- 2 delta from 1; double hashing: delta = k mod p2.
__device__ __forceinline__ uint32_t second_step(uint32_t uk, uint32_t b, uint32_t p1)
{
    uint32_t q = mod_mersenne(uk, b + 1, 2u * p1 + 1u);          // (k mod p2) mod p1
    if (q >= p1) q -= p1;
    if (q >= p1) q -= p1;
    return q;
}

template <bool SHARED, bool TRACK, typename T>
__device__ __forceinline__ void ht_accumulate_pow2(const T &tab, uint32_t mask, uint32_t b, int32_t k, typename T::Val v,
                                                   typename BestOf<typename T::Val>::type &best, unsigned &fallbacks,
                                                   uint32_t *ucnt, int32_t *ulist)
{
    const uint32_t uk = (uint32_t)k;
    const uint32_t sh = 32u - b;                       // 1 <= b <= 31
    uint32_t i = (uk * kHashMul1) >> sh;
    const uint32_t h2 = ((uk * kHashMul2) >> sh) | 1u;
    uint32_t delta = 1u;
#pragma unroll 1
    for (int t = 0; t < kMaxRetries; ++t) {
        if (try_slot<SHARED, TRACK>(tab, (size_t)i * tab.stride, k, v, best, ucnt, ulist)) return;
        i = (i + delta) & mask;
        delta = (2u * delta + h2) & mask;
    }
    ++fallbacks;
#pragma unroll 1
    for (uint32_t u = 0; u <= mask; ++u) {
        const uint32_t q = (i + u) & mask;
        if (try_slot<SHARED, TRACK>(tab, (size_t)q * tab.stride, k, v, best, ucnt, ulist)) return;
    }
}

template <bool SHARED, bool TRACK, typename T>
__device__ __forceinline__ void ht_accumulate(const T &tab, uint32_t p1, uint32_t b, int32_t k, typename T::Val v,
                                              typename BestOf<typename T::Val>::type &best, unsigned &fallbacks,
                                              uint32_t *ucnt = nullptr, int32_t *ulist = nullptr)
{
    const uint32_t uk = (uint32_t)k;
    const int mode = T::kProbe >= 0 ? T::kProbe : tab.probe;
    if (mode == kProbeQuadDoublePow2) {               // the whole 2^b allocation, mask p1
        ht_accumulate_pow2<SHARED, TRACK>(tab, p1, b, k, v, best, fallbacks, ucnt, ulist);
        return;
    }
    uint32_t i = mod_mersenne(uk, b, p1);
    uint32_t delta = (p1 > 1u) ? 1u : 0u;
    uint32_t step = 0xFFFFFFFFu;                      // (k mod p2) mod p1, on first need
    if (mode == kProbeDouble) {
        step = second_step(uk, b, p1);
        delta = step;
    }
    uint32_t s = i;
#pragma unroll 1
    for (int t = 0; t < kMaxRetries; ++t) {
        s = i;
        if (try_slot<SHARED, TRACK>(tab, (size_t)s * tab.stride, k, v, best, ucnt, ulist)) return;
        i += delta;
        if (i >= p1) i -= p1;
        if (mode == kProbeQuadDouble) {
            if (step == 0xFFFFFFFFu) step = second_step(uk, b, p1);
            unsigned long long d2 = 2ull * delta + step;    // < 3 p1
            if (d2 >= p1) d2 -= p1;
            if (d2 >= p1) d2 -= p1;
            delta = (uint32_t)d2;
        } else if (mode == kProbeQuadratic) {
            delta <<= 1;
            if (delta >= p1) delta -= p1;
        }
    }
    ++fallbacks;
#pragma unroll 1
    for (uint32_t u = 1; u <= p1; ++u) {
        uint32_t q = s + u;
        if (q >= p1) q -= p1;
        if (try_slot<SHARED, TRACK>(tab, (size_t)q * tab.stride, k, v, best, ucnt, ulist)) return;
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
    if constexpr (G == 32) {        // whole warp: two 32-bit reductions (weight word, then label word)
        const unsigned hi = (unsigned)(x >> 32);
        const unsigned mh = __reduce_max_sync(0xFFFFFFFFu, hi);
        const unsigned ml = __reduce_max_sync(0xFFFFFFFFu, hi == mh ? (unsigned)x : 0u);
        return ((unsigned long long)mh << 32) | ml;
    } else {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) x = umax64(x, __shfl_xor_sync(group_mask<G>(), x, o, G));
        return x;
    }
}

template <int G>
__device__ __forceinline__ BestD group_max(BestD x)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        BestD y;
        y.v = __shfl_xor_sync(group_mask<G>(), x.v, o, G);
        y.k = __shfl_xor_sync(group_mask<G>(), x.k, o, G);
        best_merge(x, y);
    }
    return x;
}

// Lanes of one group (G lanes, aligned inside the warp) insert their (key, weight) pairs
// into the group's shared table.  Before the per-lane inserts, up to kPeel rounds take the
// key of the lowest pending lane, sum the weights of every lane holding that key with a
// shuffle reduction and insert the sum once: after a few sweeps most neighbours of a vertex
// share a handful of labels, and same-slot atomics would otherwise serialise.  Integer
// weights keep every partial sum exact, so the table contents do not depend on the order.
constexpr int kPeel = 3;

template <int G, bool SHARED, bool TRACK, typename T>
__device__ __forceinline__ void group_insert(const T &tab, uint32_t p1, uint32_t b, bool has, int32_t k,
                                             typename T::Val w, typename BestOf<typename T::Val>::type &best,
                                             unsigned &fb, uint32_t *ucnt = nullptr, int32_t *ulist = nullptr,
                                             bool peel = true, bool unit = false, bool notab = false)
{
    using V = typename T::Val;
    if (notab) {                                       // distinct labels: the entry is its label's sum
        if (has) best_add(best, w, k);
        return;
    }
    if (G >= 2 && peel && unit) {                      // uniform over the group
        // unit weights: every group of lanes holding one label is found at once, and its lowest
        // lane inserts the group's size (its weight sum) for all of them, every group in parallel
        const unsigned same = __match_any_sync(group_mask<G>(), has ? (unsigned)k : 0xFFFFFFFFu);
        if (has && (__ffs(same) - 1) == (int)(threadIdx.x & 31))
            ht_accumulate<SHARED, TRACK>(tab, p1, b, k, V(__popc(same)), best, fb, ucnt, ulist);
        return;
    }
    if (G >= 2 && peel) {                              // uniform over the group
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
            if (lane == leader) ht_accumulate<SHARED, TRACK>(tab, p1, b, kl, sum, best, fb, ucnt, ulist);
            if (mine) has = false;
            pend &= ~same;
        }
    }
    if (has) ht_accumulate<SHARED, TRACK>(tab, p1, b, k, w, best, fb, ucnt, ulist);
}

// hashtableClear of slots [0, p1] of a contiguous, 16-byte aligned table with 16-byte stores
// (p1 + 1 is a power of two, at least 4 slots are allocated).
// (Values are cleared to all-zero bits, which is 0 for both value types.)
template <typename V, int PROBE>
__device__ __forceinline__ void clear_table_vec(const SplitTable<V, PROBE> &T, uint32_t p1, int first, int step)
{
    const uint32_t chunks = (p1 + 4u) >> 2;            // 16-byte chunks of keys (4 slots each)
    constexpr uint32_t per = sizeof(V) / sizeof(int32_t);   // value chunks per key chunk
    int4 *K4 = reinterpret_cast<int4 *>(T.k);
    int4 *V4 = reinterpret_cast<int4 *>(T.v);
    for (uint32_t q = first; q < chunks; q += step) {
        K4[q] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
#pragma unroll
        for (uint32_t r = 0; r < per; ++r) V4[q * per + r] = make_int4(0, 0, 0, 0);
    }
}

template <int PROBE>
__device__ __forceinline__ void clear_table_vec(const PackedTable<PROBE> &T, uint32_t p1, int first, int step)
{
    const uint32_t chunks = (p1 + 2u) >> 1;          // two slots per 16 bytes
    int4 *H4 = reinterpret_cast<int4 *>(T.h);
    for (uint32_t q = first; q < chunks; q += step) H4[q] = make_int4(0, kEmpty, 0, kEmpty);
}

// Clear of a thread's private interleaved table (slot s at s * stride).
// Clears slots [0, p1] (the whole 2^b allocation, which the power-of-two probe uses).
template <typename V, int PROBE>
__device__ __forceinline__ void clear_table_private(const SplitTable<V, PROBE> &T, uint32_t p1)
{
    for (uint32_t s = 0; s <= p1; ++s) {
        T.k[(size_t)s * T.stride] = kEmpty;
        T.v[(size_t)s * T.stride] = V(0);
    }
}

template <int PROBE>
__device__ __forceinline__ void clear_table_private(const PackedTable<PROBE> &T, uint32_t p1)
{
    for (uint32_t s = 0; s <= p1; ++s) T.h[(size_t)s * T.stride] = kEmptySlot;
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
    int32_t mark, pull;        // marks written this sweep; activity from moved bits (sync)
    int32_t probe;             // probe scheme of the tables
    int32_t peel;              // sum the weights of lanes holding the same label before inserting
    int32_t notab;             // every label of a row is distinct: the maximum needs no table
    int32_t pad_notab;
};

// The fields of a view read for every scanned entry (kept in registers by kernels that hold
// the full view in shared memory); load_entry and scan_row take either.
struct RowView {
    const int32_t *idx;
    const int32_t *C;
    const float *w;
    int32_t peel;
    int32_t notab;
};

__device__ __forceinline__ RowView row_of(const SweepView &a) { return RowView{a.idx, a.C, a.w, a.peel, a.notab}; }

// Marks the neighbours in entries [e0, e1) (first entry `first`, stride `step`) unprocessed for
// the next sweep.  Each thread loads kMarkUnroll indices before it stores their flags: a byte
// store may alias the index array as far as the compiler knows, so a plain loop would wait a
// full load latency per entry.
constexpr int kMarkUnroll = 8;
__device__ __forceinline__ void mark_range(uint8_t *flags, const int32_t *idx, int64_t e0, int64_t e1, int64_t first,
                                           int64_t step)
{
    for (int64_t eb = e0 + first; eb < e1; eb += kMarkUnroll * step) {
        int32_t j[kMarkUnroll];
#pragma unroll
        for (int u = 0; u < kMarkUnroll; ++u) {
            const int64_t e = eb + u * step;
            j[u] = e < e1 ? idx[e] : -1;
        }
#pragma unroll
        for (int u = 0; u < kMarkUnroll; ++u)
            if (j[u] >= 0) flags[j[u]] = 1;
    }
}

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
    v.mover_v = (l & 1) ? G.mover_v1 : G.mover_v;
    v.mover_c = G.mover_c;
    v.mover_count = G.mover_count + (l & 1);
    v.mark = rs->mark;
    v.pull = rs->pull;
    v.probe = G.probe;
    // The first sweep of a run from fresh labels (label = vertex id) finds every neighbour label
    // distinct in a duplicate-free row, so the duplicate-label rounds would find nothing there;
    // not so in an asynchronous sweep, whose labels change as it goes (by the time the hubs run,
    // most of their neighbours have moved to a few shared labels).
    v.peel = l > 0 || rs->async_mode;
    // Synchronous sweep 0 of a fresh run on rows whose indices strictly increase: every
    // neighbour label of a row is a distinct vertex id, so K_{i->c} is the weight of the one
    // entry holding c, and the arg-max of Algorithm 1 is the maximum over the entries of
    // (weight, smallest label): the kernels skip the tables.
    v.notab = (rs->fresh && l == 0 && !rs->async_mode && G.rows_strict) ? 1 : 0;
    v.pad_notab = 0;
    const int slot = (l - rs->first) % (G.ctr_iters > 0 ? G.ctr_iters : 1);
    v.ctr = G.ctr + (size_t)(slot < 0 ? 0 : slot) * kPerSweep;
    v.fallbacks = G.fallbacks;
    v.lists = G.lists;
    v.tshift = G.tshift;
    return v;
}

// Synchronous movers are staged per warp in shared memory (32 (v, c) pairs) and appended to
// the graph's mover list with one atomic per 32 movers: a per-vertex atomic on the single
// list counter would serialise in L2.  Every lane of the warp calls these; n is uniform.
__device__ __forceinline__ void movers_flush(unsigned long long *count, int32_t *mv, int32_t *mc, int2 *sbuf, int &n)
{
    if (n == 0) return;
    __syncwarp();
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(count, (unsigned long long)n);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (lane < n) {
        const int2 m = sbuf[lane];
        mv[base + lane] = m.x;
        mc[base + lane] = m.y;
    }
    __syncwarp();
    n = 0;
}

__device__ __forceinline__ void movers_push(const SweepView &a, int2 *sbuf, int &n, bool pred, int32_t v, int32_t c)
{
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, pred);
    if (!bal) return;
    const int cnt = __popc(bal);
    if (n + cnt > 32) movers_flush(a.mover_count, a.mover_v, a.mover_c, sbuf, n);
    const int lane = threadIdx.x & 31;
    if (pred) sbuf[n + __popc(bal & ((1u << lane) - 1u))] = make_int2(v, c);
    n += cnt;
}

// Loads entry e of the row of v: (label of the neighbour, weight); has = false for e past
// the row end and for self-loops (Algorithm 1 skips j = i).  With SEEN (pull sweeps) the raw
// label words are or-ed into `seen` (bit 31: the neighbour moved in the previous sweep),
// self-loops included; push sweeps never see the bit and skip that work.
template <bool SEEN, typename V, typename A>
__device__ __forceinline__ void load_entry(const A &a, int32_t v, int64_t e, int64_t end, bool &has,
                                           int32_t &k, V &wv, uint32_t &seen)
{
    has = e < end;
    k = 0;
    wv = V(0);
    if (has) {
        const int32_t j = a.idx[e];
        if (SEEN) {
            const uint32_t cj = (uint32_t)a.C[j];
            seen |= cj;
            has = (j != v);
            k = (int32_t)(cj & kLabelMask);
            if (has) wv = a.w ? to_value<V>(a.w[e]) : V(1);
        } else {
            has = (j != v);
            if (has) {
                k = a.C[j];
                wv = a.w ? to_value<V>(a.w[e]) : V(1);
            }
        }
    }
}

// Scans entries [start, end) of the row of v in rounds: each round covers U * step entries,
// lane offset `lane` inside each step.  All U entries of a round are loaded (index, weight,
// gathered label) before any of them is inserted, so U gathers per thread are in flight.
template <int G, bool SHARED, bool TRACK, int U, bool SEEN, typename T, typename A>
__device__ __forceinline__ void scan_row(const A &a, int32_t v, int64_t start, int64_t end, int step,
                                         int lane, const T &tab, uint32_t p1, uint32_t b,
                                         typename BestOf<typename T::Val>::type &best, unsigned &fb,
                                         uint32_t &seen, uint32_t *ucnt = nullptr, int32_t *ulist = nullptr,
                                         int round = 0)
{
    using V = typename T::Val;
    const int64_t adv = round ? round : (int64_t)step * U;   // a block-wide round for the CTA kernels
    for (int64_t eb = start; eb < end; eb += adv) {
        bool has[U];
        int32_t k[U];
        V wv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) load_entry<SEEN>(a, v, eb + (int64_t)u * step + lane, end, has[u], k[u], wv[u], seen);
#pragma unroll
        for (int u = 0; u < U; ++u)
            group_insert<G, SHARED, TRACK>(tab, p1, b, has[u], k[u], wv[u], best, fb, ucnt, ulist, a.peel != 0,
                                           a.w == nullptr, a.notab != 0);
    }
}

// Move rule of Algorithm 1: c* != C[i] and, on Pick-Less sweeps, c* < C[i].
__device__ __forceinline__ bool decide(unsigned long long best, int32_t cur, int pl, int32_t &cstar)
{
    if (best == 0) return false;                   // no neighbour label (isolated / self-loops only)
    cstar = unpack_key(best);
    return (cstar != cur) && (!pl || cstar < cur);
}

__device__ __forceinline__ bool decide(const BestD &best, int32_t cur, int pl, int32_t &cstar)
{
    if (best.k < 0) return false;
    cstar = best.k;
    return (cstar != cur) && (!pl || cstar < cur);
}

// Shared-memory tables use the packed layout when the sums are integers.
constexpr bool kPackShared = true;
template <typename V, bool PACK, int PROBE> struct TableFor {
    using type = SplitTable<V, PROBE>;
};
template <int PROBE> struct TableFor<uint32_t, true, PROBE> {
    using type = PackedTable<PROBE>;
};

// Table t of n_tables tables of `slots` slots at `base` (8 bytes per slot in both layouts):
// interleaved (slot s of table t at s * n_tables + t) or one table after another.
template <typename V, int PROBE>
__device__ __forceinline__ void table_at(SplitTable<V, PROBE> &T, unsigned char *base, int n_tables, int slots, int t,
                                         bool interleaved)
{
    V *vbase = (V *)(base + (size_t)n_tables * slots * sizeof(int32_t));
    if (interleaved) {
        T.k = (int32_t *)base + t;
        T.v = vbase + t;
        T.stride = n_tables;
    } else {
        T.k = (int32_t *)base + (size_t)t * slots;
        T.v = vbase + (size_t)t * slots;
        T.stride = 1;
    }
}

template <int PROBE>
__device__ __forceinline__ void table_at(PackedTable<PROBE> &T, unsigned char *base, int n_tables, int slots, int t,
                                         bool interleaved)
{
    if (interleaved) {
        T.h = (unsigned long long *)base + t;
        T.stride = n_tables;
    } else {
        T.h = (unsigned long long *)base + (size_t)t * slots;
        T.stride = 1;
    }
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

// Entries loaded per lane and round by the G-lane kernels: for G = 1 and G = 8 enough that one
// round covers the default degree range of the bucket (D <= 8, D <= 32), so a row's index,
// weight and label loads are all in flight together; for G = 32 two (64 entries a round),
// which with four resident blocks per SM measured faster than four entries with three blocks.
constexpr int kUnrollThread = 2;      // G = 1
constexpr int kUnrollSmall = 4;       // G = 2, 4
constexpr int kUnrollGroup = 2;       // G = 8, 16
constexpr int kUnrollWarp = 2;        // G = 32
constexpr int kMinBlocksThread = 8;   // resident blocks per SM asked of the register allocator (128 threads)
constexpr int kMinBlocks = 4;         // (256 threads)
template <int G> struct GroupUnroll {
    static constexpr int U = G == 1 ? kUnrollThread : (G <= 4 ? kUnrollSmall : (G <= 16 ? kUnrollGroup : kUnrollWarp));
    static constexpr int kMinBlocks = G == 1 ? ::lpa::kMinBlocksThread : ::lpa::kMinBlocks;
};

// G lanes per vertex (G = 1: thread per vertex with a private table; G = 32: warp per
// vertex).  Persistent: each warp takes work items (a range of one graph's bucket list) from
// the queue.  The warp fetches the list entry, processed flag and row bounds of 32 vertices
// at once (one per lane), then its groups take them 32/G at a time: the per-vertex chain of
// dependent loads (list, flag, offsets) is paid once per 32 vertices.  Neighbour ids of a
// row that fits one round stay in registers for the marks.
template <int G, int TPB, typename V, bool PULL, int PROBE>
__global__ void __launch_bounds__(TPB, GroupUnroll<G>::kMinBlocks) k_group(KArgs k)
{
    if (*k.active == 0) return;                        // every graph has stopped
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NG = TPB / G;
    constexpr int GPW = 32 / G;                        // groups per warp
    constexpr int U = GroupUnroll<G>::U;
    const int lane_w = threadIdx.x & 31;
    const int lane = (G == 1) ? 0 : (threadIdx.x & (G - 1));
    const int grp = threadIdx.x / G;
    const int gw = lane_w / G;                         // group within the warp
    using Tab = typename TableFor<V, kPackShared, PROBE>::type;
    Tab tab;
    if (G == 1) table_at(tab, smem, TPB, k.slots, threadIdx.x, true);      // private, interleaved
    else table_at(tab, smem, NG, k.slots, grp, false);
    __shared__ int2 s_mov[TPB / 32][32];
    int2 *mbuf = s_mov[threadIdx.x >> 5];
    int nmov = 0;
    // counters and movers are kept per warp while consecutive items belong to one graph
    int cur_g = -1;
    // The graph's view lives in shared memory, one per warp (its many pointers would otherwise
    // hold registers across the scan); the three read for every entry are kept in registers.
    __shared__ SweepView s_view[TPB / 32];
    SweepView &a = s_view[threadIdx.x >> 5];
    const int32_t *a_idx = nullptr, *a_C = nullptr;
    const float *a_w = nullptr;
    bool notab = false;
    unsigned fb = 0, c_act = 0, c_edges = 0, c_moved = 0, c_marks = 0;
    for (;;) {
        int it = 0;
        if (lane_w == 0) it = (int)atomicAdd(k.queue, 1u);
        it = __shfl_sync(0xFFFFFFFFu, it, 0);
        if (it >= k.n_items) break;
        const WorkItem item = k.items[it];
        if (item.g != cur_g) {
            if (cur_g >= 0) {
                movers_flush(a.mover_count, a.mover_v, a.mover_c, mbuf, nmov);
                warp_flush(a, k.kslot, c_act, c_edges, c_moved, c_marks, fb);
                fb = c_act = c_edges = c_moved = c_marks = 0;
            }
            cur_g = item.g;
            __syncwarp();
            if (lane_w == 0) a = view_of(k.gd, item.g);
            __syncwarp();
            a_idx = a.idx;
            a_C = a.C;
            a_w = a.w;
            notab = a.notab != 0;
            tab.probe = a.probe;
        }
        if (a.done || (a.pull != 0) != PULL) continue;                // the other launch takes it
        for (int64_t base = 0; base < item.count; base += 32) {       // uniform per warp
            // lane L: vertex base + L of the item (its flag is taken here: mark processed; in a
            // pull sweep every vertex is a candidate and its activity is known after the scan)
            int32_t mv = -1;
            int64_t mo0 = 0, mo1 = 0;
            if (base + lane_w < item.count) {
                mv = __ldg(a.lists + item.start + base + lane_w);
                bool cand = PULL;
                if (!PULL && a.flag_cur[mv] != 0) {
                    a.flag_cur[mv] = 0;
                    cand = true;
                }
                if (cand) {
                    mo0 = a.off[mv];
                    mo1 = a.off[mv + 1];
                } else {
                    mv = -1;                                   // not active in this sweep
                }
            }
#pragma unroll 1
            for (int st = 0; st < 32 && base + st < item.count; st += GPW) {    // uniform per warp
                const int src = st + gw;
                const int32_t v = __shfl_sync(0xFFFFFFFFu, mv, src);
                const int64_t o0 = __shfl_sync(0xFFFFFFFFu, mo0, src);
                const int64_t o1 = __shfl_sync(0xFFFFFFFFu, mo1, src);
                const bool cand = v >= 0 && o1 > o0;
                int32_t cstar = -1;
                bool moved = false;
                if (cand) {
                    const uint32_t D = (uint32_t)(o1 - o0);
                    const uint32_t b = cap_bits(D << a.tshift);    // capacity >= D << tshift
                    const uint32_t p1 = cap_of_bits(b);
                    const int32_t cur = PULL ? (int32_t)((uint32_t)a.C[v] & kLabelMask) : a.C[v];
                    uint32_t seen = 0;
                    if (notab) {
                    } else if (G == 1) {
                        clear_table_private(tab, p1);              // hashtableClear
                    } else {
                        group_sync<G>();                           // previous vertex's inserts are done
                        clear_table_vec(tab, p1, lane, G);
                        group_sync<G>();
                    }
                    typename BestOf<V>::type best;
                    best_init(best);
                    int32_t jr[U];                                 // neighbour ids of the first round
#pragma unroll
                    for (int u = 0; u < U; ++u) jr[u] = -1;
                    for (int64_t eb = o0; eb < o1; eb += (int64_t)U * G) {
                        bool has[U];
                        int32_t kk[U];
                        V wv[U];
#pragma unroll
                        for (int u = 0; u < U; ++u) {              // indices and weights
                            const int64_t e = eb + (int64_t)u * G + lane;
                            has[u] = e < o1;
                            jr[u] = has[u] ? a_idx[e] : -1;
                            wv[u] = (has[u] && a_w) ? to_value<V>(a_w[e]) : V(1);
                        }
#pragma unroll
                        for (int u = 0; u < U; ++u) {              // labels (self-loops not inserted)
                            if (PULL) {
                                const uint32_t cj = has[u] ? (uint32_t)a_C[jr[u]] : 0u;
                                seen |= cj;
                                has[u] = has[u] && jr[u] != v;
                                kk[u] = (int32_t)(cj & kLabelMask);
                            } else {
                                has[u] = has[u] && jr[u] != v;
                                kk[u] = has[u] ? a_C[jr[u]] : 0;
                            }
                        }
                        // inserts one slot at a time (rolled loop, entries shifted down in
                        // registers) so that the probe loop is not replicated U times
#pragma unroll 1
                        for (int u = 0; u < U; ++u) {
                            if (!__any_sync(group_mask<G>(), has[0])) break;     // lanes of this group only
                            group_insert<G, (G > 1), false>(tab, p1, b, has[0], kk[0], wv[0], best, fb, nullptr,
                                                            nullptr, a.peel != 0, a_w == nullptr, notab);
#pragma unroll
                            for (int q = 0; q + 1 < U; ++q) {
                                has[q] = has[q + 1];
                                kk[q] = kk[q + 1];
                                wv[q] = wv[q + 1];
                            }
                            has[U - 1] = false;
                        }
                    }
                    best = group_max<G>(best);                     // hashtableMaxKey
                    bool act = true;
                    if (PULL) {                                    // a neighbour moved in the last sweep
                        if (G > 1) seen = __reduce_or_sync(group_mask<G>(), seen);
                        act = (seen & kMovedBit) != 0;
                    }
                    moved = act && decide(best, cur, a.pl, cstar);
                    if (moved) {
                        if (a.async_mode && lane == 0) {
                            a.C[v] = cstar;
                            __threadfence();
                        }
                        if (!a.mark) {
                        } else if (D <= (uint32_t)(U * G)) {       // mark neighbours (ids in registers)
#pragma unroll
                            for (int u = 0; u < U; ++u)
                                if (jr[u] >= 0) a.flag_next[jr[u]] = 1;
                        } else {
                            mark_range(a.flag_next, a_idx, o0, o1, lane, G);
                        }
                    }
                    if (lane == 0 && act) {
                        c_act += 1;
                        c_edges += D;
                        if (moved) {
                            c_moved += 1;
                            c_marks += D;                  // entries of the movers
                        }
                    }
                }
                if (!a.async_mode) movers_push(a, mbuf, nmov, moved && lane == 0, v, cstar);
            }
        }
    }
    if (cur_g >= 0) {
        movers_flush(a.mover_count, a.mover_v, a.mover_c, mbuf, nmov);
        warp_flush(a, k.kslot, c_act, c_edges, c_moved, c_marks, fb);
    }
}

// ---------------------------------------------------------------------------------
// Low-degree buckets (thread, group and warp by default): a warp per batch of vertices, with
// the batch's rows flattened.  The warp fetches the list entry, processed flag and row bounds
// of 32 vertices at once, packs as many of them as fit its shared-memory region into a
// sub-batch (each vertex gets its own table of 2^b slots, 2^b - 1 >= D << tshift), and then
// scans the sub-batch's rows as one run of entries: in each round lane L takes flat entry
// f0 + L, finds its vertex (segment) from a bit mask of the segment starts in the round's
// window (one warp reduction per 32 entries), and inserts the neighbour label into that
// vertex's table.  Every lane has an entry in every round but the last, whatever the
// degrees.  A lane's running maximum (sum << 32 | ~label) is folded into its segment's
// shared maximum when its entries pass into the next segment.  Then one lane per vertex
// takes the decision of Algorithm 1.  Integer weights keep every sum exact, so the tables
// and the decisions do not depend on which lane adds first.
constexpr int kFlatWarps = 8;            // warps per block (256 threads)
constexpr int kFlatMinSlots = 1024;      // table slots per warp region (8 bytes each) at least
constexpr int kFlatU = 2;                // 32-entry windows per round (loads in flight per lane)

__device__ __forceinline__ unsigned lanemask_le()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

template <typename V, int PROBE>
__device__ __forceinline__ void flat_table(SplitTable<V, PROBE> &T, unsigned char *region, int wslots, uint32_t tb)
{
    T.k = (int32_t *)region + tb;
    T.v = (V *)(region + (size_t)wslots * sizeof(int32_t)) + tb;
    T.stride = 1;
}

template <int PROBE>
__device__ __forceinline__ void flat_table(PackedTable<PROBE> &T, unsigned char *region, int, uint32_t tb)
{
    T.h = (unsigned long long *)region + tb;
    T.stride = 1;
}

// Clears slots [0, total) of a warp region with 16-byte stores (rounded up to whole stores;
// the region's slot count is a multiple of 4).
template <typename V, int PROBE>
__device__ __forceinline__ void flat_clear(const SplitTable<V, PROBE> &, unsigned char *region, int wslots, uint32_t total,
                                           int lane)
{
    int4 *K4 = reinterpret_cast<int4 *>(region);
    int4 *V4 = reinterpret_cast<int4 *>(region + (size_t)wslots * sizeof(int32_t));
    constexpr uint32_t per = sizeof(V) / sizeof(int32_t);
    for (uint32_t q = lane; q < ((total + 3u) >> 2); q += 32) {        // the region holds whole 4-slot groups
        K4[q] = make_int4(kEmpty, kEmpty, kEmpty, kEmpty);
#pragma unroll
        for (uint32_t r = 0; r < per; ++r) V4[q * per + r] = make_int4(0, 0, 0, 0);
    }
}

template <int PROBE>
__device__ __forceinline__ void flat_clear(const PackedTable<PROBE> &, unsigned char *region, int, uint32_t total, int lane)
{
    int4 *H4 = reinterpret_cast<int4 *>(region);
    for (uint32_t q = lane; q < ((total + 1u) >> 1); q += 32) H4[q] = make_int4(0, kEmpty, 0, kEmpty);
}

template <typename V, bool PULL, int PROBE>
__global__ void __launch_bounds__(kFlatWarps * 32, 3) k_flat(KArgs k)
{
    if (*k.active == 0) return;                        // every graph has stopped
    extern __shared__ __align__(16) unsigned char smem[];
    using Tab = typename TableFor<V, kPackShared, PROBE>::type;
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int wslots = k.slots;                        // slots per warp region
    unsigned char *region = smem + (size_t)wid * wslots * 8;
    __shared__ long long s_eoff[kFlatWarps][32];       // row start minus the segment's first flat index
    __shared__ int32_t s_vtx[kFlatWarps][32];          // vertex of each segment
    __shared__ uint32_t s_tab[kFlatWarps][32];         // table base slot << 5 | b
    __shared__ unsigned long long s_best[kFlatWarps][32];
    __shared__ int32_t s_seen[kFlatWarps][32];
    __shared__ int2 s_mov[kFlatWarps][32];
    int2 *mbuf = s_mov[wid];
    int nmov = 0;
    int cur_g = -1;
    SweepView a{};
    Tab tab;
    unsigned fb = 0, c_act = 0, c_edges = 0, c_moved = 0, c_marks = 0;
    for (;;) {
        int it = 0;
        if (lane == 0) it = (int)atomicAdd(k.queue, 1u);
        it = __shfl_sync(0xFFFFFFFFu, it, 0);
        if (it >= k.n_items) break;
        const WorkItem item = k.items[it];
        if (item.g != cur_g) {
            if (cur_g >= 0) {
                movers_flush(a.mover_count, a.mover_v, a.mover_c, mbuf, nmov);
                warp_flush(a, k.kslot, c_act, c_edges, c_moved, c_marks, fb);
                fb = c_act = c_edges = c_moved = c_marks = 0;
            }
            cur_g = item.g;
            a = view_of(k.gd, item.g);
            tab.probe = a.probe;
        }
        if (a.done || (a.pull != 0) != PULL) continue;                // the other launch takes it
        for (int64_t base = 0; base < item.count; base += 32) {       // uniform per warp
            // lane L: vertex base + L of the item, its flag taken (push sweeps), its row
            int32_t v = -1, cur = 0;
            int64_t o0 = 0;
            uint32_t D = 0;
            if (base + lane < item.count) {
                v = __ldg(a.lists + item.start + base + lane);
                bool cand = PULL;
                if (!PULL && a.flag_cur[v] != 0) {
                    a.flag_cur[v] = 0;                 // mark processed
                    cand = true;
                }
                if (cand) {
                    o0 = a.off[v];
                    D = (uint32_t)(a.off[v + 1] - o0);
                    cur = PULL ? (int32_t)((uint32_t)a.C[v] & kLabelMask) : a.C[v];
                }
            }
            // the launcher sizes the region for the bucket's largest degree, so cap <= wslots
            const uint32_t b = D ? cap_bits(D << a.tshift) : 0u;
            const uint32_t cap = D ? (1u << b) : 0u;
            const uint32_t cincl = warp_incl_scan(cap);
            uint32_t consumed = 0;                     // slots of the earlier sub-batches
            bool handled = (D == 0);
#pragma unroll 1
            while (true) {                             // uniform per warp
                const bool in = !handled && (cincl - consumed <= (uint32_t)wslots);
                const unsigned mask = __ballot_sync(0xFFFFFFFFu, in);
                if (mask == 0) break;                  // every vertex of the batch is done
                const int ci = __popc(mask & lanemask_lt());           // segment index
                const uint32_t Dm = in ? D : 0u;
                const uint32_t dincl = warp_incl_scan(Dm);
                const uint32_t start = dincl - Dm;                     // first flat entry of the segment
                const int last = 31 - __clz(mask);
                const uint32_t E = __shfl_sync(0xFFFFFFFFu, dincl, last);
                const uint32_t total = __shfl_sync(0xFFFFFFFFu, cincl, last) - consumed;
                if (in) {
                    s_eoff[wid][ci] = (long long)o0 - (long long)start;
                    s_vtx[wid][ci] = v;
                    s_tab[wid][ci] = ((cincl - cap - consumed) << 5) | b;
                    s_best[wid][ci] = 0ull;
                    s_seen[wid][ci] = 0;
                }
                flat_clear(tab, region, wslots, total, lane);            // hashtableClear of every table
                __syncwarp();
                unsigned long long best = 0ull;
                int bseg = 0;                          // segment of `best`
                uint32_t before = 0;                   // segment starts below the round's window
#pragma unroll 1
                for (uint32_t f0 = 0; f0 < E; f0 += 32 * kFlatU) {
                    bool has[kFlatU];
                    int seg[kFlatU];
                    int32_t kk[kFlatU];
                    V wv[kFlatU];
                    int64_t ee[kFlatU];
                    int32_t jj[kFlatU];
#pragma unroll
                    for (int u = 0; u < kFlatU; ++u) {                   // segment of each entry
                        const uint32_t w0 = f0 + 32u * u;
                        const unsigned bit = (in && start >= w0 && start < w0 + 32u) ? (1u << (start - w0)) : 0u;
                        const unsigned M = __reduce_or_sync(0xFFFFFFFFu, bit);
                        seg[u] = (int)(before + __popc(M & lanemask_le())) - 1;
                        before += __popc(M);
                        has[u] = w0 + lane < E;
                        ee[u] = has[u] ? s_eoff[wid][seg[u]] + (long long)(w0 + lane) : 0;
                    }
#pragma unroll
                    for (int u = 0; u < kFlatU; ++u) {                   // indices and weights
                        jj[u] = has[u] ? a.idx[ee[u]] : 0;
                        wv[u] = (has[u] && a.w) ? to_value<V>(a.w[ee[u]]) : V(1);
                    }
#pragma unroll
                    for (int u = 0; u < kFlatU; ++u) {                   // labels (self-loops not inserted)
                        if (PULL) {
                            const uint32_t cj = has[u] ? (uint32_t)a.C[jj[u]] : 0u;
                            if (cj & kMovedBit) s_seen[wid][seg[u]] = 1;
                            kk[u] = (int32_t)(cj & kLabelMask);
                        } else {
                            kk[u] = has[u] ? a.C[jj[u]] : 0;
                        }
                        has[u] = has[u] && jj[u] != s_vtx[wid][seg[u]];
                    }
                    // inserts (sg, key, w) into segment sg's table, folding the lane's maximum of the
                    // previous segment into that segment's shared maximum first
                    auto insert = [&](int sg, int32_t key, V w) {
                        if (sg != bseg) {
                            if (best) atomicMax(&s_best[wid][bseg], best);
                            best = 0ull;
                            bseg = sg;
                        }
                        const uint32_t tw = s_tab[wid][sg];
                        const uint32_t bb = tw & 31u;
                        Tab t = tab;
                        flat_table(t, region, wslots, tw >> 5);
                        ht_accumulate<true, false>(t, cap_of_bits(bb), bb, key, w, best, fb);
                    };
#pragma unroll 1
                    for (int u = 0; u < kFlatU; ++u) {
                        // lanes holding the same label of the same segment: the lowest inserts their
                        // summed weight once (up to kPeel labels per step): after the first sweeps most
                        // neighbours of a vertex share a few labels, and same-slot atomics serialise
                        if (a.peel && a.w == nullptr) {          // unit weights: all label groups at once
                            // lanes with the same label and the same segment: two 32-bit matches
                            const unsigned same = __match_any_sync(0xFFFFFFFFu, has[0] ? (uint32_t)kk[0] : 0xFFFFFFFFu) &
                                                  __match_any_sync(0xFFFFFFFFu, (uint32_t)seg[0]);
                            if (has[0] && (__ffs(same) - 1) == lane) insert(seg[0], kk[0], V(__popc(same)));
                            has[0] = false;
                        }
                        unsigned pend = __ballot_sync(0xFFFFFFFFu, has[0]);
#pragma unroll 1
                        for (int r = 0; r < kPeel && pend && a.peel; ++r) {
                            const int leader = __ffs(pend) - 1;
                            const int32_t kl = __shfl_sync(0xFFFFFFFFu, kk[0], leader);
                            const int sl = __shfl_sync(0xFFFFFFFFu, seg[0], leader);
                            const bool mine = has[0] && kk[0] == kl && seg[0] == sl;
                            const unsigned same = __ballot_sync(0xFFFFFFFFu, mine);
                            if (__popc(same) < 2) break;
                            V sum = mine ? wv[0] : V(0);
                            if constexpr (std::is_same<V, uint32_t>::value) {
                                sum = __reduce_add_sync(0xFFFFFFFFu, sum);
                            } else {
#pragma unroll
                                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
                            }
                            if (lane == leader) insert(sl, kl, sum);
                            if (mine) has[0] = false;
                            pend &= ~same;
                        }
                        if (has[0]) insert(seg[0], kk[0], wv[0]);
#pragma unroll
                        for (int q = 0; q + 1 < kFlatU; ++q) {
                            has[q] = has[q + 1];
                            seg[q] = seg[q + 1];
                            kk[q] = kk[q + 1];
                            wv[q] = wv[q + 1];
                        }
                        has[kFlatU - 1] = false;
                    }
                }
                if (best) atomicMax(&s_best[wid][bseg], best);
                __syncwarp();
                // one lane per vertex: the move rule of Algorithm 1
                int32_t cstar = -1;
                bool moved = false;
                if (in) {
                    const unsigned long long bw = s_best[wid][ci];
                    const bool act = PULL ? (s_seen[wid][ci] != 0) : true;
                    moved = act && decide(bw, cur, a.pl, cstar);
                    if (act) {
                        c_act += 1;
                        c_edges += D;
                    }
                    if (moved) {
                        c_moved += 1;
                        c_marks += D;                  // entries of the movers
                        if (a.async_mode) {
                            a.C[v] = cstar;
                            __threadfence();
                        }
                    }
                }
                if (!a.async_mode) movers_push(a, mbuf, nmov, moved, v, cstar);
                if (a.mark) {                          // mark the movers' neighbours
                    unsigned mm = __ballot_sync(0xFFFFFFFFu, moved);
                    while (mm) {
                        const int src = __ffs(mm) - 1;
                        mm &= mm - 1;
                        const int64_t r0 = __shfl_sync(0xFFFFFFFFu, o0, src);
                        const uint32_t rd = __shfl_sync(0xFFFFFFFFu, D, src);
                        mark_range(a.flag_next, a.idx, r0, r0 + rd, lane, 32);
                    }
                }
                __syncwarp();                          // the region and the segment data are free
                consumed = __shfl_sync(0xFFFFFFFFu, cincl, last);
                handled = handled || in;
            }
        }
    }
    if (cur_g >= 0) {
        movers_flush(a.mover_count, a.mover_v, a.mover_c, mbuf, nmov);
        warp_flush(a, k.kslot, c_act, c_edges, c_moved, c_marks, fb);
    }
}

// Resident blocks per SM asked of the register allocator for the block tiers: 32 warps per SM
// (64 registers a thread); the 128-thread tier otherwise took 94 registers and ran 20 warps
// per SM (R-MAT 26: that tier 30 % faster with 32).
template <int TPB> constexpr int kCtaMinBlocks() { return TPB <= 128 ? 8 : (TPB <= 256 ? 4 : (TPB <= 512 ? 2 : 1)); }

// One thread block per vertex; the table (up to k.slots entries) lives in dynamic smem.
// Persistent: each block takes work items from the queue; the list entries, processed flags
// and row bounds of up to 32 vertices of the item are fetched at once into shared memory.
// A vertex costs two block barriers: after its scan, every warp takes the block's maximum
// from the warps' maxima and decides the move itself (no barrier waits for one thread's
// decision) and the block clears the slots the vertex used; the second barrier waits for the
// clear, so the table is clean when the next vertex starts.
template <int TPB, typename V, bool PULL, int PROBE>
__global__ void __launch_bounds__(TPB, kCtaMinBlocks<TPB>()) k_cta(KArgs k)
{
    if (*k.active == 0) return;
    constexpr int NW = TPB / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    using Tab = typename TableFor<V, kPackShared, PROBE>::type;
    Tab tab;
    table_at(tab, smem, 1, k.slots, 0, false);
    __shared__ int s_item, s_nmov;
    __shared__ int32_t s_mv[32];
    __shared__ int64_t s_mo0[32], s_mo1[32];
    __shared__ int2 s_mov[32];
    using Best = typename BestOf<V>::type;
    __shared__ Best s_best[NW];                        // the warps' maxima
    __shared__ unsigned long long s_mbase;
    if (threadIdx.x == 0) s_nmov = 0;
    clear_table_vec(tab, (uint32_t)k.slots - 1u, threadIdx.x, TPB);   // clean at the start
    // counters (thread 0) are kept while consecutive items belong to one graph
    int cur_g = -1;
    // The graph's view lives in shared memory (its pointers would otherwise hold registers
    // across the scan); the fields read for every entry are kept in registers.
    __shared__ SweepView s_view;
    SweepView &a = s_view;
    RowView r{};
    unsigned fb = 0;
    unsigned long long c_act = 0, c_edges = 0, c_moved = 0, c_marks = 0;
    auto flush_counts = [&]() {
        if (threadIdx.x == 0) {
            unsigned long long *c = a.ctr + k.kslot * kCtrFields;
            if (c_act) atomicAdd(c + CTR_ACTIVE, c_act);
            if (c_edges) atomicAdd(c + CTR_EDGES, c_edges);
            if (c_moved) atomicAdd(c + CTR_MOVED, c_moved);
            if (c_marks) atomicAdd(c + CTR_MARKS, c_marks);
        }
        if (fb) atomicAdd(a.fallbacks, (unsigned long long)fb);
        fb = 0;
        c_act = c_edges = c_moved = c_marks = 0;
    };
    for (;;) {
        __syncthreads();                               // s_item of the last round is consumed
        if (threadIdx.x == 0) s_item = (int)atomicAdd(k.queue, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= k.n_items) break;
        const WorkItem item = k.items[it];
        if (item.g != cur_g) {                         // uniform for the block
            if (cur_g >= 0) flush_counts();
            cur_g = item.g;
            __syncthreads();                           // the last graph's view is no longer read
            if (threadIdx.x == 0) a = view_of(k.gd, item.g);
            __syncthreads();
            r = row_of(a);
        }
        if (a.done || (a.pull != 0) != PULL) continue;        // the other launch takes it
        for (int64_t base = 0; base < item.count; base += 32) {
            __syncthreads();                           // the previous batch is finished
            if (threadIdx.x < 32 && base + threadIdx.x < item.count) {
                int32_t v0 = __ldg(a.lists + item.start + base + threadIdx.x);
                int64_t m0 = 0, m1 = 0;
                bool cand = PULL;                      // pull sweep: activity known after the scan
                if (!PULL && a.flag_cur[v0] != 0) {
                    a.flag_cur[v0] = 0;                // mark processed
                    cand = true;
                }
                if (cand) {
                    m0 = a.off[v0];
                    m1 = a.off[v0 + 1];
                } else {
                    v0 = -1;
                }
                s_mv[threadIdx.x] = v0;
                s_mo0[threadIdx.x] = m0;
                s_mo1[threadIdx.x] = m1;
            }
            __syncthreads();
            const int nb = (int)(item.count - base < 32 ? item.count - base : 32);
            for (int q = 0; q < nb; ++q) {
                const int32_t v = s_mv[q];
                if (v < 0) continue;                   // uniform for the block
                const int64_t o0 = s_mo0[q], o1 = s_mo1[q];
                const uint32_t D = (uint32_t)(o1 - o0);
                const uint32_t b = cap_bits(D << a.tshift);
                const uint32_t p1 = cap_of_bits(b);
                const int32_t cur = PULL ? (int32_t)((uint32_t)r.C[v] & kLabelMask) : r.C[v];
                tab.probe = a.probe;                   // the table is clean: cleared after its last use
                Best best;
                best_init(best);
                uint32_t seen = 0;
                constexpr int U = 2;                           // loads in flight per thread
                scan_row<32, true, false, U, PULL>(r, v, o0 + (threadIdx.x & ~31) * U, o1, 32, threadIdx.x & 31, tab,
                                                   p1, b, best, fb, seen, nullptr, nullptr, TPB * U);
                best = group_max<32>(best);
                if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
                bool act = true;
                if (PULL) act = __syncthreads_or((seen & kMovedBit) != 0) != 0;   // a neighbour moved
                else __syncthreads();
                // the scan is over: every warp combines the maxima and decides; the slots of
                // this vertex are cleared
                Best x;
                best_init(x);
                if ((threadIdx.x & 31) < NW) x = s_best[threadIdx.x & 31];
                x = group_max<32>(x);
                int32_t cstar = -1;
                const bool moved = act && decide(x, cur, a.pl, cstar);
                if (!r.notab) clear_table_vec(tab, p1, threadIdx.x, TPB);
                if (moved) {
                    if (threadIdx.x == 0) {
                        if (a.async_mode) {
                            a.C[v] = cstar;
                            __threadfence();
                        } else {
                            s_mov[s_nmov++] = make_int2(v, cstar);     // at most 32 per batch
                        }
                    }
                    if (a.async_mode) __syncthreads();
                    if (a.mark)
                        mark_range(a.flag_next, r.idx, o0, o1, threadIdx.x, TPB);
                }
                if (threadIdx.x == 0 && act) {
                    c_act += 1;
                    c_edges += D;
                    if (moved) {
                        c_moved += 1;
                        c_marks += D;                  // entries of the movers
                    }
                }
                __syncthreads();                       // the table is clean for the next vertex
            }
            // append the batch's synchronous movers with one atomic
            __syncthreads();
            const int nm = s_nmov;
            if (nm > 0) {
                if (threadIdx.x == 0) s_mbase = atomicAdd(a.mover_count, (unsigned long long)nm);
                __syncthreads();
                if (threadIdx.x < nm) {
                    const int2 m = s_mov[threadIdx.x];
                    a.mover_v[s_mbase + threadIdx.x] = m.x;
                    a.mover_c[s_mbase + threadIdx.x] = m.y;
                }
                __syncthreads();
                if (threadIdx.x == 0) s_nmov = 0;
            }
        }
    }
    if (cur_g >= 0) flush_counts();
}

// ---------------------------------------------------------------------------------
// Hubs: tables in HBM shared by several blocks.  Per sweep: begin (take the processed
// flag), accumulate (a block per CSR chunk; each block folds its running maximum into
// hub_best), clear (a block per slice of the used-slot list or of the table), move (the
// decision), mark (a block per CSR chunk of the hubs that moved).  Items: begin and move take
// a graph's hubs [start, start + count); accumulate, clear and mark take one chunk / slice.
// Whether graph g's hubs take the two passes in this sweep: every sweep (hub_tp = 2), or only
// in the first sweep of a run from fresh labels (hub_tp = 1), where every neighbour label of a
// duplicate-free row is distinct and the HBM tables' atomics miss the most; later sweeps,
// with few labels left, are cheaper in the single pass.  With hub_tp = 1 a sweep that needs no
// tables (notab) takes the single pass, which then only takes the maximum (with hub_tp = 2
// the single-pass chunks do not exist).
__device__ __forceinline__ bool hub_two_pass_now(const GraphDev &G, const SweepView &a)
{
    return G.hub_tp == 2 || (G.hub_tp == 1 && !a.peel && !a.notab);
}

struct HArgs {
    const GraphDev *gd;
    const WorkItem *items;
    const int32_t *active;
    int32_t chunk;
    int32_t pad;
};

// Slots taken from empty are collected in a block-local list in shared memory and copied to
// the hub's used list with one global atomic per block.  A graph with integer sums keeps its
// hub tables in the packed layout, any other graph in the split float layout.
// The block's arg-max is folded into hub_best with one atomic maximum (packed word), or, for
// float64 sums, stored as the chunk's pair and reduced over the hub's chunks by k_hub_move.
template <int TPB, bool PULL, typename T>
__device__ __forceinline__ void hub_accumulate(const SweepView &a, const HubArgs &h, int hh, int64_t c, const T &tab,
                                               int32_t *s_list, uint32_t &s_cnt, uint32_t &s_base,
                                               typename BestOf<typename T::Val>::type *s_best)
{
    const int32_t v = h.hub_v[hh];
    const uint32_t p1 = h.hub_p1[hh], b = h.hub_b[hh];
    const int64_t e0 = h.chunk_e0[c], e1 = h.chunk_e1[c];
    unsigned fb = 0;
    typename BestOf<typename T::Val>::type best;
    best_init(best);
    uint32_t seen = 0;
    scan_row<32, true, true, 2, PULL>(row_of(a), v, e0 + (threadIdx.x & ~31) * 2, e1, 32, threadIdx.x & 31, tab, p1, b,
                                      best, fb, seen, &s_cnt, s_list, TPB * 2);
    if (fb) atomicAdd(a.fallbacks, (unsigned long long)fb);
    best = group_max<32>(best);
    if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
    if (PULL) {
        if (__syncthreads_or((seen & kMovedBit) != 0) && threadIdx.x == 0) h.hub_seen[hh] = 1;
    } else {
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int w = 1; w < TPB / 32; ++w) best_merge(best, s_best[w]);
        if constexpr (std::is_same<typename T::Val, double>::value) {
            h.chunk_bv[c] = best.v;
            h.chunk_bk[c] = best.k;
        } else {
            if (best) atomicMax(h.hub_best + hh, best);
        }
        s_base = s_cnt ? atomicAdd(h.hub_used + hh, s_cnt) : 0u;
    }
    __syncthreads();
    int32_t *ulist = h.used_list + h.used_base[hh] + s_base;
    for (uint32_t q = threadIdx.x; q < s_cnt; q += TPB) ulist[q] = s_list[q];
}

template <int TPB, bool PULL, int PROBE, bool F64>
__global__ void __launch_bounds__(TPB, 2) k_hub_acc(HArgs k)
{
    if (*k.active == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t *s_list = (int32_t *)smem;                 // [chunk]
    __shared__ typename BestOf<typename std::conditional<F64, double, float>::type>::type s_best[TPB / 32];
    __shared__ uint32_t s_cnt, s_base;
    const WorkItem item = k.items[blockIdx.x];
    __shared__ SweepView s_view;                       // in shared memory: frees registers for the scan
    if (threadIdx.x == 0) s_view = view_of(k.gd, item.g);
    __syncthreads();
    const SweepView &a = s_view;
    if (a.done || (a.pull != 0) != PULL) return;      // the other launch takes it
    if (hub_two_pass_now(k.gd[item.g], a)) return;    // the two-pass kernels take this sweep
    const HubArgs &h = k.gd[item.g].hub;
    const int64_t c = item.start;
    const int hh = h.chunk_h[c];
    if (!h.hub_act[hh]) return;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    if constexpr (F64) {
        SplitTable<double, PROBE> tab{h.tab_k + h.hub_tab[hh], h.tab_vd + h.hub_tab[hh], 1, a.probe};
        hub_accumulate<TPB, PULL>(a, h, hh, c, tab, s_list, s_cnt, s_base, s_best);
    } else if (k.gd[item.g].int_weights) {
        PackedTable<PROBE, true> tab{(unsigned long long *)h.tab_k + h.hub_tab[hh], 1, a.probe};
        hub_accumulate<TPB, PULL>(a, h, hh, c, tab, s_list, s_cnt, s_base, s_best);
    } else {
        SplitTable<float, PROBE> tab{h.tab_k + h.hub_tab[hh], h.tab_v + h.hub_tab[hh], 1, a.probe};
        hub_accumulate<TPB, PULL>(a, h, hh, c, tab, s_list, s_cnt, s_base, s_best);
    }
}

// Two-pass accumulation of hubs with integer label sums (packed slots) and HBM tables.
//
// Pass 1 (k_hub_part, a block per kPartChunk-entry chunk of a hub's row): the chunk's labels
// are summed in a shared-memory table (Algorithm 2's accumulate), then every distinct (label,
// sum) pair of the chunk goes to label partition part(label) of the hub: a block-wide count
// per partition, one global reservation per partition, and the pairs written to the
// partition's buffer.  Pass 2 (k_hub_merge, a block per partition): the partition's pairs are
// summed in a shared-memory table, whose running maximum (sum << 32 | ~label) is folded into
// the hub's maximum.  Every pair of one label goes to the same partition, so a partition's
// table holds the label's whole sum K_{i->c}, and the hub's maximum over its partitions is the
// arg-max of Algorithm 1 with the smallest label on ties, as in the single-pass tables.
// Instead of round-tripping the hub tables through DRAM with global atomics, the sweep streams
// the pairs once out and once in.  A partition whose reservations pass kPartCap overflows: its
// pairs beyond the cap go to the hub's HBM table at once, and pass 2 sends the buffered ones
// there too, so that each label's sum is whole in one place.
constexpr int kPartThreads = 512;
constexpr uint32_t kPartTableBits = 13;              // 8192 slots: load <= 1/2 for a full chunk
constexpr uint32_t kHashMul3 = 0xC2B2AE3Du;          // odd multiplier of the partition hash

__device__ __forceinline__ uint32_t part_of(int32_t k, uint32_t pb)
{
    return pb ? (((uint32_t)k * kHashMul3) >> (32u - pb)) : 0u;
}


// Sends (label, sum) to its partition: a reserved position below kPartCap, else the hub's HBM
// table (and the partition is marked overflowed).
template <int PROBE>
__device__ __forceinline__ void part_put(const HubArgs &h, const SweepView &a, int hh, int32_t pbase,
                                         const uint32_t *s_base, uint32_t *s_fill, uint32_t part, int32_t key,
                                         uint32_t sum, unsigned long long &obest, unsigned &fb)
{
    const uint32_t pos = s_base[part] + atomicAdd(&s_fill[part], 1u);
    if (pos < (uint32_t)kPartCap) {
        h.pairs[(size_t)(pbase + part) * kPartCap + pos] = ((unsigned long long)(uint32_t)key << 32) | sum;
    } else {
        h.part_ovf[pbase + part] = 1;
        const PackedTable<PROBE, true> htab{(unsigned long long *)h.tab_k + h.hub_tab[hh], 1, a.probe};
        ht_accumulate<true, true>(htab, h.hub_p1[hh], h.hub_b[hh], key, sum, obest, fb, h.hub_used + hh,
                                  h.used_list + h.used_base[hh]);
    }
}

// Pass 1.  Blocks loop over the first-pass chunks.  In a sweep on fresh labels (no duplicate
// grouping) the chunk's entries go to the partitions as they are; otherwise the chunk's
// labels are first summed in a shared-memory table and its distinct pairs go.
template <bool PULL, int PROBE>
__global__ void __launch_bounds__(kPartThreads, 2) k_hub_part(HArgs k, int32_t n_items, int32_t one_graph)
{
    if (*k.active == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *T = (unsigned long long *)smem;                 // [2^kPartTableBits]
    uint32_t *s_cnt = (uint32_t *)(smem + ((size_t)8 << kPartTableBits)); // [2^kPartMaxBits] counts, then fill
    uint32_t *s_base = s_cnt + (1 << kPartMaxBits);                       // [2^kPartMaxBits] reservations
    constexpr int PER = kPartChunk / kPartThreads;                        // entries per thread (8)
    int skip_g = -1;                                   // a graph whose hubs take the single pass now
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {            // uniform per block
        const WorkItem item = k.items[it];
        if (item.g == skip_g) continue;
        const GraphDev &G = k.gd[item.g];
        const SweepView a = view_of(k.gd, item.g);
        if (a.done || (a.pull != 0) != PULL || !hub_two_pass_now(G, a)) {
            if (one_graph) return;                     // every item belongs to this graph
            skip_g = item.g;
            continue;
        }
        const HubArgs &h = G.hub;
        const int64_t c = item.start;
        const int hh = h.pc_h[c];
        if (!h.hub_act[hh]) continue;
        const int32_t v = h.hub_v[hh];
        const int64_t e0 = h.pc_e0[c], e1 = h.pc_e1[c];
        const uint32_t pb = h.hub_pb[hh], np = 1u << pb;
        const int32_t pbase = h.hub_pbase[hh];
        __syncthreads();                               // the previous item's shared data is consumed
        for (uint32_t q = threadIdx.x; q < np; q += kPartThreads) s_cnt[q] = 0;
        unsigned fb = 0;
        unsigned long long obest = 0ull;               // overflow inserts into the HBM table
        uint32_t seen = 0;
        if (!a.peel) {
            // the entries themselves: count per partition, reserve, write
            int32_t key[PER];
            uint32_t wsum[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int64_t e = e0 + threadIdx.x + (int64_t)u * kPartThreads;
                key[u] = -1;
                wsum[u] = 0;
                if (e < e1) {
                    const int32_t j = a.idx[e];
                    if (j != v) wsum[u] = a.w ? (uint32_t)a.w[e] : 1u;
                    key[u] = j;                        // neighbour id first; its label below
                    if (j == v) key[u] = -1;
                }
            }
            uint32_t cj[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) cj[u] = key[u] >= 0 ? (uint32_t)a.C[key[u]] : 0u;   // all gathers in flight
            __syncthreads();                           // s_cnt cleared
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                if (key[u] < 0) continue;
                if (PULL) seen |= cj[u];
                key[u] = (int32_t)(cj[u] & kLabelMask);
                atomicAdd(&s_cnt[part_of(key[u], pb)], 1u);
            }
            __syncthreads();
            for (uint32_t q = threadIdx.x; q < np; q += kPartThreads) {
                const uint32_t n = s_cnt[q];
                s_base[q] = n ? atomicAdd(h.part_cnt + pbase + q, n) : 0u;
                s_cnt[q] = 0;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < PER; ++u)
                if (key[u] >= 0)
                    part_put<PROBE>(h, a, hh, pbase, s_base, s_cnt, part_of(key[u], pb), key[u], wsum[u], obest, fb);
        } else {
            // the chunk's labels summed first, then its distinct pairs
            constexpr uint32_t b = kPartTableBits;
            const uint32_t p1 = cap_of_bits(b);
            const PackedTable<PROBE> tab{T, 1, a.probe};
            clear_table_vec(tab, p1, threadIdx.x, kPartThreads);
            __syncthreads();
            unsigned long long best = 0ull;            // (not used: pass 2 takes the maximum)
            scan_row<32, true, false, 2, PULL>(a, v, e0 + (threadIdx.x & ~31) * 2, e1, 32, threadIdx.x & 31, tab,
                                               p1, b, best, fb, seen, nullptr, nullptr, kPartThreads * 2);
            __syncthreads();
            for (uint32_t q = threadIdx.x; q <= p1; q += kPartThreads) {
                const unsigned long long x = T[q];
                if ((uint32_t)(x >> 32) != 0xFFFFFFFFu) atomicAdd(&s_cnt[part_of((int32_t)(x >> 32), pb)], 1u);
            }
            __syncthreads();
            for (uint32_t q = threadIdx.x; q < np; q += kPartThreads) {
                const uint32_t n = s_cnt[q];
                s_base[q] = n ? atomicAdd(h.part_cnt + pbase + q, n) : 0u;
                s_cnt[q] = 0;
            }
            __syncthreads();
            for (uint32_t q = threadIdx.x; q <= p1; q += kPartThreads) {
                const unsigned long long x = T[q];
                const int32_t key = (int32_t)(x >> 32);
                if (key != kEmpty)
                    part_put<PROBE>(h, a, hh, pbase, s_base, s_cnt, part_of(key, pb), key, (uint32_t)x, obest, fb);
            }
        }
        if (PULL && __syncthreads_or((seen & kMovedBit) != 0) && threadIdx.x == 0) h.hub_seen[hh] = 1;
        if (obest) atomicMax(h.hub_best + hh, obest);
        if (fb) atomicAdd(a.fallbacks, (unsigned long long)fb);
    }
}

// Pass 2.  Blocks loop over the partitions: each partition's pairs summed in a shared-memory
// table (or, after an overflow, all of them in the hub's HBM table), the running maximum
// folded into the hub's; the partition's counters are reset for the next sweep.
template <int PROBE>
__global__ void __launch_bounds__(kPartThreads, 3) k_hub_merge(HArgs k, int32_t n_items, int32_t one_graph)
{
    if (*k.active == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_best[kPartThreads / 32];
    __shared__ uint32_t s_n;
    __shared__ int32_t s_ovf;
    int skip_g = -1;                                   // a graph whose hubs take the single pass now
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {            // uniform per block
        const WorkItem item = k.items[it];
        if (item.g == skip_g) continue;
        const GraphDev &G = k.gd[item.g];
        const SweepView a = view_of(k.gd, item.g);
        if (a.done || !hub_two_pass_now(G, a)) {
            if (one_graph) return;                     // every item belongs to this graph
            skip_g = item.g;
            continue;
        }
        const HubArgs &h = G.hub;
        const int32_t q = (int32_t)item.start;
        const int hh = h.part_h[q];
        __syncthreads();                               // the previous item's shared data is consumed
        if (threadIdx.x == 0) {
            const uint32_t c = h.part_cnt[q];
            s_n = c < (uint32_t)kPartCap ? c : (uint32_t)kPartCap;
            s_ovf = h.part_ovf[q];
            h.part_cnt[q] = 0;                         // ready for the next sweep
            h.part_ovf[q] = 0;
        }
        __syncthreads();
        const uint32_t n = s_n;
        if (n == 0) continue;
        const unsigned long long *P = h.pairs + (size_t)q * kPartCap;
        unsigned fb = 0;
        unsigned long long best = 0ull;
        if (!s_ovf) {
            uint32_t b = cap_bits(n << 1);
            if (b > kPartTableBits) b = kPartTableBits;
            const uint32_t p1 = cap_of_bits(b);
            const PackedTable<PROBE> tab{(unsigned long long *)smem, 1, a.probe};
            clear_table_vec(tab, p1, threadIdx.x, kPartThreads);
            __syncthreads();
            for (uint32_t i0 = threadIdx.x & ~31u; i0 < n; i0 += kPartThreads) {     // uniform per warp
                const uint32_t i = i0 + (threadIdx.x & 31u);
                const bool has = i < n;
                const unsigned long long x = has ? P[i] : 0ull;
                group_insert<32, true, false>(tab, p1, b, has, (int32_t)(x >> 32), (uint32_t)x, best, fb, nullptr,
                                              nullptr, a.peel != 0);
            }
        } else {                                       // the partition overflowed: all of it to HBM
            const PackedTable<PROBE, true> htab{(unsigned long long *)h.tab_k + h.hub_tab[hh], 1, a.probe};
            for (uint32_t i = threadIdx.x; i < n; i += kPartThreads) {
                const unsigned long long x = P[i];
                ht_accumulate<true, true>(htab, h.hub_p1[hh], h.hub_b[hh], (int32_t)(x >> 32), (uint32_t)x, best, fb,
                                          h.hub_used + hh, h.used_list + h.used_base[hh]);
            }
        }
        best = group_max<32>(best);
        if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kPartThreads / 32; ++w) best = umax64(best, s_best[w]);
            if (best) atomicMax(h.hub_best + hh, best);
        }
        if (fb) atomicAdd(a.fallbacks, (unsigned long long)fb);
    }
}

// Hubs whose table fits in the shared memory of a cluster of CS blocks (1024 threads each).
// Persistent: rank 0 takes a hub from the queue and broadcasts it; every block clears its
// slice of the hub's table, the cluster synchronises, every block scans 1/CS of the row and
// inserts into the distributed table (Algorithm 2's probe sequence over the whole table),
// folds its running maximum into hub_best, and the cluster synchronises again before the
// next hub.  Integer sums only (packed slots).
constexpr int kDsmThreads = 1024;

template <int CS, bool PULL, int PROBE>
__global__ void __cluster_dims__(CS, 1, 1) __launch_bounds__(kDsmThreads) k_hub_dsm(HArgs k, int32_t n_items,
                                                                                   unsigned *queue)
{
    if (*k.active == 0) return;                        // the same value in every block of the cluster
    cg::cluster_group cluster = cg::this_cluster();
    const unsigned rank = cluster.block_rank();
    constexpr int csb = CS == 2 ? 1 : (CS == 4 ? 2 : (CS == 8 ? 3 : 4));
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *slice = (unsigned long long *)smem;
    __shared__ int s_it;
    __shared__ unsigned long long s_best[kDsmThreads / 32];
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const int it = (int)atomicAdd(queue, 1u);
            for (unsigned r = 0; r < (unsigned)CS; ++r) *cluster.map_shared_rank(&s_it, r) = it;
        }
        cluster.sync();                                // the hub is known in every block
        const int it = s_it;
        if (it >= n_items) break;
        const WorkItem item = k.items[it];
        const SweepView a = view_of(k.gd, item.g);
        const HubArgs &h = k.gd[item.g].hub;
        const int hh = (int)item.start;
        if (a.done || (a.pull != 0) != PULL || !h.hub_act[hh]) {
            cluster.sync();                            // s_it is read before rank 0 writes the next
            continue;
        }
        const uint32_t b = h.hub_b[hh], p1 = h.hub_p1[hh];
        const uint32_t lb = b - csb;                   // 2^lb slots per block
        clear_table_vec(PackedTable<PROBE>{slice, 1}, (1u << lb) - 1u, threadIdx.x, kDsmThreads);
        cluster.sync();                                // every slice is clear
        const ClusterTable<PROBE> tab{slice, lb, 1, a.probe};
        const int32_t v = h.hub_v[hh];
        const int64_t o0 = a.off[v], o1 = a.off[v + 1];
        const int64_t per = (o1 - o0 + CS - 1) / CS;
        const int64_t e0 = o0 + (int64_t)rank * per;
        const int64_t e1 = e0 + per < o1 ? e0 + per : o1;
        unsigned fb = 0;
        unsigned long long best = 0;
        uint32_t seen = 0;
        if (e0 < e1)
            scan_row<32, true, false, 2, PULL>(a, v, e0 + (threadIdx.x & ~31) * 2, e1, 32, threadIdx.x & 31, tab,
                                               p1, b, best, fb, seen, nullptr, nullptr, kDsmThreads * 2);
        if (fb) atomicAdd(a.fallbacks, (unsigned long long)fb);
        best = group_max<32>(best);
        if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
        bool any_seen = false;
        if (PULL) any_seen = __syncthreads_or((seen & kMovedBit) != 0) != 0;
        else __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < kDsmThreads / 32; ++w) best = umax64(best, s_best[w]);
            if (best) atomicMax(h.hub_best + hh, best);
            if (PULL && any_seen) h.hub_seen[hh] = 1;
        }
        cluster.sync();                                // every insert is done before the next clear
    }
}

// ---------------------------------------------------------------------------------
// launchers

static int g_num_sms = 0;       // per translation unit
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


// Dynamic shared memory beyond the default allowance: the kernels' own static shared memory
// (at most a few KB) counts against the same 48 KB, hence the margin.
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 40 * 1024) return cudaSuccess;
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

template <int G, int TPB, typename V, bool PULL, int PROBE>
static cudaError_t launch_gv(const KArgs &k, cudaStream_t s)
{
    constexpr int NG = TPB / G;
    const size_t smem = (size_t)NG * k.slots * (sizeof(int32_t) + sizeof(V));
    cudaError_t e = set_smem(k_group<G, TPB, V, PULL, PROBE>, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = persistent_grid(k_group<G, TPB, V, PULL, PROBE>, TPB, smem, ((int64_t)k.n_items + 7) / 8 * 8);
    k_group<G, TPB, V, PULL, PROBE><<<(unsigned)(blocks < 1 ? 1 : blocks), TPB, smem, s>>>(k);
    return cudaGetLastError();
}

template <typename V, bool PULL, int PROBE>
static cudaError_t launch_flat(const KArgs &k0, cudaStream_t s)
{
    KArgs k = k0;
    k.slots = k.slots > kFlatMinSlots ? k.slots : kFlatMinSlots;     // a region holds the bucket's largest table
    const size_t smem = (size_t)kFlatWarps * k.slots * 8;
    cudaError_t e = set_smem(k_flat<V, PULL, PROBE>, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = persistent_grid(k_flat<V, PULL, PROBE>, kFlatWarps * 32, smem,
                                           ((int64_t)k.n_items + kFlatWarps - 1) / kFlatWarps);
    k_flat<V, PULL, PROBE><<<(unsigned)(blocks < 1 ? 1 : blocks), kFlatWarps * 32, smem, s>>>(k);
    return cudaGetLastError();
}

// Value type of the tables: double with F64 (lpa_tuning.float_values = 2), else uint32 for
// integer sums and float for the rest.
template <int G, int TPB, bool PULL, int PROBE, bool F64>
static cudaError_t launch_g(const KArgs &k, bool int_w, cudaStream_t s)
{
    if constexpr (F64) return launch_gv<G, TPB, double, PULL, PROBE>(k, s);
    else return int_w ? launch_gv<G, TPB, uint32_t, PULL, PROBE>(k, s) : launch_gv<G, TPB, float, PULL, PROBE>(k, s);
}

template <int TPB, typename V, bool PULL, int PROBE>
static cudaError_t launch_cv(const KArgs &k, cudaStream_t s)
{
    const size_t smem = (size_t)k.slots * (sizeof(int32_t) + sizeof(V));
    cudaError_t e = set_smem(k_cta<TPB, V, PULL, PROBE>, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = persistent_grid(k_cta<TPB, V, PULL, PROBE>, TPB, smem, k.n_items);
    k_cta<TPB, V, PULL, PROBE><<<(unsigned)(blocks < 1 ? 1 : blocks), TPB, smem, s>>>(k);
    return cudaGetLastError();
}

template <int TPB, bool PULL, int PROBE, bool F64>
static cudaError_t launch_cvt(const KArgs &k, bool int_w, cudaStream_t s)
{
    if constexpr (F64) return launch_cv<TPB, double, PULL, PROBE>(k, s);
    else return int_w ? launch_cv<TPB, uint32_t, PULL, PROBE>(k, s) : launch_cv<TPB, float, PULL, PROBE>(k, s);
}

template <bool PULL, int PROBE, bool F64>
static cudaError_t launch_cta(const KArgs &k, int threads, bool int_w, cudaStream_t s)
{
    switch (threads) {
    case 64: return launch_cvt<64, PULL, PROBE, F64>(k, int_w, s);
    case 128: return launch_cvt<128, PULL, PROBE, F64>(k, int_w, s);
    case 256: return launch_cvt<256, PULL, PROBE, F64>(k, int_w, s);
    case 512: return launch_cvt<512, PULL, PROBE, F64>(k, int_w, s);
    case 1024: return launch_cvt<1024, PULL, PROBE, F64>(k, int_w, s);
    default: return cudaErrorInvalidValue;
    }
}

// The kernel of bucket b for the push (PULL = false) or pull sweeps of the plan's graphs;
// each instantiation has its own work-queue counter.
template <bool PULL, int PROBE, bool F64>
static cudaError_t launch_vertex(const SweepPlan &p, int b, cudaStream_t s)
{
    KArgs k{};
    k.gd = p.gd;
    k.items = p.items[b];
    k.n_items = p.n_items[b];
    k.slots = p.slots[b];
    k.queue = p.queues + b + (PULL ? B_COUNT : 0);
    k.active = p.active_count;
    k.kslot = b;                                       // bucket index == kernel slot
    const bool iw = p.int_weights != 0;
    if (!F64 && b <= B_WARP && ((p.flat_buckets >> b) & 1))   // flattened rows, a warp per batch of vertices
        return iw ? launch_flat<uint32_t, PULL, PROBE>(k, s) : launch_flat<float, PULL, PROBE>(k, s);
    switch (b) {
    case B_THREAD: return launch_g<1, 128, PULL, PROBE, F64>(k, iw, s);
    case B_GROUP:
        switch (p.group_lanes) {
        case 2: return launch_g<2, 256, PULL, PROBE, F64>(k, iw, s);
        case 4: return launch_g<4, 256, PULL, PROBE, F64>(k, iw, s);
        case 8: return launch_g<8, 256, PULL, PROBE, F64>(k, iw, s);
        case 16: return launch_g<16, 256, PULL, PROBE, F64>(k, iw, s);
        default: return cudaErrorInvalidValue;
        }
    case B_WARP: return launch_g<32, 256, PULL, PROBE, F64>(k, iw, s);
    case B_CTA: return launch_cta<PULL, PROBE, F64>(k, p.cta_threads, iw, s);
    case B_CTA_LARGE: return launch_cta<PULL, PROBE, F64>(k, p.cta_large_threads, iw, s);
    case B_CTA_XL: return launch_cta<PULL, PROBE, F64>(k, p.cta_xl_threads, iw, s);
    default: return cudaErrorInvalidValue;
    }
}

constexpr size_t kDsmSmem = ((size_t)1 << kDsmSliceBits) * sizeof(unsigned long long);

template <int CS, bool PULL, int PROBE>
static cudaError_t launch_dsm_cs(const HArgs &h, int32_t n_items, unsigned *queue, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(k_hub_dsm<CS, PULL, PROBE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDsmSmem);
    if (e == cudaSuccess && CS > 8)
        e = cudaFuncSetAttribute(k_hub_dsm<CS, PULL, PROBE>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    query_device();
    int64_t clusters = g_num_sms / CS;
    if (clusters > n_items) clusters = n_items;
    if (clusters < 1) clusters = 1;
    k_hub_dsm<CS, PULL, PROBE><<<(unsigned)(clusters * CS), kDsmThreads, kDsmSmem, s>>>(h, n_items, queue);
    return cudaGetLastError();
}

// Cluster class c (cluster of 2 << c blocks).
template <bool PULL, int PROBE>
static cudaError_t launch_dsm(int c, const HArgs &h, int32_t n_items, unsigned *queue, cudaStream_t s)
{
    switch (c) {
    case 0: return launch_dsm_cs<2, PULL, PROBE>(h, n_items, queue, s);
    case 1: return launch_dsm_cs<4, PULL, PROBE>(h, n_items, queue, s);
    case 2: return launch_dsm_cs<8, PULL, PROBE>(h, n_items, queue, s);
    case 3: return launch_dsm_cs<16, PULL, PROBE>(h, n_items, queue, s);
    default: return cudaErrorInvalidValue;
    }
}

// The table kernels of one sweep for probe scheme PROBE: every vertex bucket, then (after
// k_hub_begin, which the caller launches) the hub accumulation in HBM or cluster tables.
// Push and pull variants as the plan asks; CUDA-event hooks per kernel slot.
template <int PROBE, bool F64 = false>
static cudaError_t launch_vertex_phase(const SweepPlan &p, cudaStream_t s, LaunchHook *hook, int *launches)
{
    const bool push = p.pull_mode != 1, pull = p.pull_mode != 0;
    for (int b = B_THREAD; b <= B_CTA_XL; ++b) {
        if (p.n_items[b] <= 0) continue;
        if (hook) hook->before(b);
        cudaError_t r = push ? launch_vertex<false, PROBE, F64>(p, b, s) : cudaSuccess;
        if (r == cudaSuccess && pull) r = launch_vertex<true, PROBE, F64>(p, b, s);
        if (hook) hook->after(b);
        if (r != cudaSuccess) return r;
        if (launches) *launches += (push ? 1 : 0) + (pull ? 1 : 0);
    }
    return cudaSuccess;
}

// Persistent grid of the two-pass hub kernels: `per_sm` 512-thread blocks per SM.
static unsigned part_grid(int32_t n_items, int per_sm)
{
    query_device();
    const int64_t cap = (int64_t)g_num_sms * per_sm;
    return (unsigned)(n_items < cap ? (n_items < 1 ? 1 : n_items) : cap);
}

template <int PROBE, bool F64 = false>
static cudaError_t launch_hub_acc_phase(const SweepPlan &p, const HArgs &h, cudaStream_t s, LaunchHook *hook,
                                        int *launches)
{
    const bool push = p.pull_mode != 1, pull = p.pull_mode != 0;
    if (hook) hook->before(LPA_K_HUB_ACC);
    cudaError_t r = cudaSuccess;
    if (p.n_hub_items[HL_ACC] > 0) {                  // hubs with tables in HBM
        HArgs ha = h;
        ha.items = p.hub_items[HL_ACC];
        const size_t smem = (size_t)p.hub_chunk * sizeof(int32_t);
        if (push && r == cudaSuccess) {
            r = set_smem(k_hub_acc<1024, false, PROBE, F64>, smem);
            if (r == cudaSuccess) k_hub_acc<1024, false, PROBE, F64><<<p.n_hub_items[HL_ACC], 1024, smem, s>>>(ha);
            if (launches) ++*launches;
        }
        if (pull && r == cudaSuccess) {
            r = set_smem(k_hub_acc<1024, true, PROBE, F64>, smem);
            if (r == cudaSuccess) k_hub_acc<1024, true, PROBE, F64><<<p.n_hub_items[HL_ACC], 1024, smem, s>>>(ha);
            if (launches) ++*launches;
        }
    }
    if (!F64 && p.n_hub_items[HL_PACC] > 0 && r == cudaSuccess) {     // two-pass hubs
        HArgs ha = h;
        ha.items = p.hub_items[HL_PACC];
        const size_t smem_a = ((size_t)8 << kPartTableBits) + 2 * sizeof(uint32_t) * ((size_t)1 << kPartMaxBits);
        if (push && r == cudaSuccess) {
            r = set_smem(k_hub_part<false, PROBE>, smem_a);
            if (r == cudaSuccess)
                k_hub_part<false, PROBE><<<part_grid(p.n_hub_items[HL_PACC], 2), kPartThreads, smem_a, s>>>(
                    ha, p.n_hub_items[HL_PACC], p.n_graphs == 1);
            if (launches) ++*launches;
        }
        if (pull && r == cudaSuccess) {
            r = set_smem(k_hub_part<true, PROBE>, smem_a);
            if (r == cudaSuccess)
                k_hub_part<true, PROBE><<<part_grid(p.n_hub_items[HL_PACC], 2), kPartThreads, smem_a, s>>>(
                    ha, p.n_hub_items[HL_PACC], p.n_graphs == 1);
            if (launches) ++*launches;
        }
        if (r == cudaSuccess && p.n_hub_items[HL_PMERGE] > 0) {
            ha.items = p.hub_items[HL_PMERGE];
            const size_t smem_b = (size_t)8 << kPartTableBits;
            r = set_smem(k_hub_merge<PROBE>, smem_b);
            if (r == cudaSuccess)
                k_hub_merge<PROBE><<<part_grid(p.n_hub_items[HL_PMERGE], 3), kPartThreads, smem_b, s>>>(
                    ha, p.n_hub_items[HL_PMERGE], p.n_graphs == 1);
            if (launches) ++*launches;
        }
    }
    for (int c = 0; c < 4 && r == cudaSuccess; ++c) {    // hubs with tables in cluster memory
        if (p.n_hub_items[HL_DSM2 + c] <= 0) continue;
        HArgs ha = h;
        ha.items = p.hub_items[HL_DSM2 + c];
        if (push) {
            r = launch_dsm<false, PROBE>(c, ha, p.n_hub_items[HL_DSM2 + c], p.queues + 2 * B_COUNT + c, s);
            if (launches) ++*launches;
        }
        if (pull && r == cudaSuccess) {
            r = launch_dsm<true, PROBE>(c, ha, p.n_hub_items[HL_DSM2 + c], p.queues + 2 * B_COUNT + 4 + c, s);
            if (launches) ++*launches;
        }
    }
    if (r == cudaSuccess) r = cudaGetLastError();
    if (hook) hook->after(LPA_K_HUB_ACC);
    return r;
}

// Defined in lpa_sweep_alt.cu (the run-time probe scheme instantiation).
cudaError_t sweep_init_constants_alt();
cudaError_t launch_vertex_phase_alt(const SweepPlan &p, cudaStream_t s, LaunchHook *hook, int *launches);
cudaError_t launch_hub_acc_phase_alt(const SweepPlan &p, const HArgs &h, cudaStream_t s, LaunchHook *hook,
                                     int *launches);
// Defined in lpa_sweep_f64.cu (float64 table values, both probe instantiations).
cudaError_t sweep_init_constants_f64();
cudaError_t launch_vertex_phase_f64(const SweepPlan &p, cudaStream_t s, LaunchHook *hook, int *launches);
cudaError_t launch_hub_acc_phase_f64(const SweepPlan &p, const HArgs &h, cudaStream_t s, LaunchHook *hook,
                                     int *launches);

}  // namespace lpa
