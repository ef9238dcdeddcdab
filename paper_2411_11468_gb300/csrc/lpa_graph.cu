// Host side of liblpa.so: graph handles, validation, degree buckets, the iteration loop of
// Algorithm 1 (lpa), label/state access and the float64 modularity reduction (Eq. 1).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <mutex>

#include <algorithm>
#include <climits>
#include <type_traits>
#include <cmath>
#include <string>
#include <vector>

#include "lpa_graph_internal.h"

namespace lpa {

static thread_local std::string t_error;
void set_error(const std::string &msg) { t_error = msg; }

}  // namespace lpa

using namespace lpa;

namespace {

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

// ------------------------------------------------------------------------------------
// kernels used at creation, initialisation and for modularity

__global__ void k_off32to64(const int32_t *in, int64_t *out, int64_t n1)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i];
}

// error bits: 1 offsets decrease, 2 offsets[0] != 0, 4 offsets[n] != m, 8 index out of
// range, 16 weight negative / NaN / Inf.  Also counts the adjacent index pairs that do not
// increase, over the whole index array (desc[0]) and where the second entry starts a
// non-empty row (desc[1]): every row's indices strictly increase iff the two are equal.
__global__ void k_validate(const int64_t *off, const int32_t *idx, const float *w, int64_t n, int64_t m,
                           unsigned *err, unsigned long long *desc)
{
    unsigned bad = 0;
    unsigned long long d_all = 0, d_row = 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        if (off[0] != 0) bad |= 2u;
        if (off[n] != m) bad |= 4u;
    }
    for (int64_t i = tid; i < n; i += stride) {
        const int64_t b = off[i], b1 = off[i + 1];
        if (b > b1) bad |= 1u;
        if (i > 0 && b > 0 && b < m && b1 > b && idx[b - 1] >= idx[b]) ++d_row;
    }
    for (int64_t e = tid; e < m; e += stride) {
        const int32_t j = idx[e];
        if (j < 0 || (int64_t)j >= n) bad |= 8u;
        if (e + 1 < m && j >= idx[e + 1]) ++d_all;
        if (w) {
            const float x = w[e];
            if (!(isfinite(x) && x >= 0.0f)) bad |= 16u;
        }
    }
    if (bad) atomicOr(err, bad);
    if (d_all) atomicAdd(desc + 0, d_all);
    if (d_row) atomicAdd(desc + 1, d_row);
}

__device__ __forceinline__ unsigned long long mix_sym(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Undirectedness check: multiset of (min, max, weight) over entries with i < j must equal
// the one over entries with i > j; compared through wrapping sums of a 64-bit hash.
__global__ void k_symmetric(const int64_t *off, const int32_t *idx, const float *w, int64_t n,
                            unsigned long long *acc)
{
    unsigned long long lo = 0, hi = 0, clo = 0, chi = 0;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        for (int64_t e = off[i] + lane; e < off[i + 1]; e += 32) {
            const int64_t j = idx[e];
            if (j == i) continue;
            const unsigned long long a = (unsigned long long)(i < j ? i : j), b = (unsigned long long)(i < j ? j : i);
            const unsigned wb = w ? __float_as_uint(w[e]) : 0x3F800000u;
            const unsigned long long h = mix_sym((a << 32 | b) + 0x9E3779B97F4A7C15ull) ^ mix_sym(wb + 0x632BE59BD9B4E019ull);
            if (i < j) { lo += h; ++clo; } else { hi += h; ++chi; }
        }
    }
    atomicAdd(acc + 0, lo);
    atomicAdd(acc + 1, hi);
    atomicAdd(acc + 2, clo);
    atomicAdd(acc + 3, chi);
}

__device__ __forceinline__ int bucket_of(int64_t D, const lpa_tuning &t)
{
    if (D <= 0) return -1;
    if (D <= t.thread_max) return B_THREAD;
    if (D <= t.group_max) return B_GROUP;
    if (D <= t.warp_max) return B_WARP;
    if (D <= t.cta_max) return B_CTA;
    if (D <= t.cta_large_max) return B_CTA_LARGE;
    if (D <= t.cta_xl_max) return B_CTA_XL;
    return B_HUB;
}

// per tile of 1024 vertices: how many fall in each bucket
__global__ void __launch_bounds__(1024) k_bucket_count(const int64_t *off, int64_t n, lpa_tuning t, int32_t *cnt)
{
    __shared__ int32_t s[B_COUNT];
    if (threadIdx.x < B_COUNT) s[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    if (i < n) {
        const int b = bucket_of(off[i + 1] - off[i], t);
        if (b >= 0) atomicAdd(&s[b], 1);
    }
    __syncthreads();
    if (threadIdx.x < B_COUNT) cnt[blockIdx.x * B_COUNT + threadIdx.x] = s[threadIdx.x];
}

// stable fill: vertices of a tile keep ascending order inside each bucket list
__global__ void __launch_bounds__(1024) k_bucket_fill(const int64_t *off, int64_t n, lpa_tuning t,
                                                      const int64_t *base, int32_t *lists)
{
    __shared__ int32_t wcnt[B_COUNT][32];
    const int64_t i = blockIdx.x * 1024ll + threadIdx.x;
    const int b = (i < n) ? bucket_of(off[i + 1] - off[i], t) : -1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned my_rank = 0;
    for (int q = 0; q < B_COUNT; ++q) {
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, b == q);
        if (b == q) my_rank = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) wcnt[q][warp] = __popc(bal);
    }
    __syncthreads();
    if (b >= 0) {
        int64_t pos = base[blockIdx.x * B_COUNT + b];
        for (int w2 = 0; w2 < warp; ++w2) pos += wcnt[b][w2];
        lists[pos + my_rank] = (int32_t)i;
    }
}

__global__ void k_gather_rows(const int32_t *vs, int64_t k, const int64_t *off, int64_t *o0, int64_t *o1)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < k) {
        o0[t] = off[vs[t]];
        o1[t] = off[vs[t] + 1];
    }
}

__global__ void k_init_labels(const int64_t *off, int64_t n, int32_t *C, uint8_t *flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        C[i] = (int32_t)i;
        flag[i] = off[i + 1] > off[i] ? 1 : 0;
    }
}

// set_state: check labels, sanitise flags (vertices without edges are never processed)
__global__ void k_check_state(const int64_t *off, int64_t n, const int32_t *C, uint8_t *flag, unsigned *err)
{
    unsigned bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (C[i] < 0 || (int64_t)C[i] >= n) bad = 1;
        if (flag) flag[i] = (flag[i] != 0 && off[i + 1] > off[i]) ? 1 : 0;
    }
    if (bad) atomicOr(err, bad);
}

__device__ __forceinline__ double warp_sum_d(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

// Eq. 1 numerators: Sigma_c = sum of K_i over i in c is pre-aggregated per block in a small
// shared-memory table and added to the global Sigma with one atomic per distinct label per
// block (one label may cover most of the graph, and per-vertex atomics on it would
// serialise); labels that do not fit go to Sigma directly.
constexpr int kModSlots = 1024;

template <typename ACC>
__device__ __forceinline__ void mod_sigma_add_t(int32_t *sk, ACC *sv, ACC *Sig, int32_t c, ACC k)
{
    uint32_t s = ((uint32_t)c * 2654435761u) >> 22;
    for (int t = 0; t < 8; ++t, s = (s + 1) & (kModSlots - 1)) {
        int32_t kk = *((volatile int32_t *)(sk + s));
        if (kk == -1) {
            const int32_t old = atomicCAS(sk + s, -1, c);
            kk = (old == -1) ? c : old;
        }
        if (kk == c) {
            atomicAdd(sv + s, k);
            return;
        }
    }
    atomicAdd(Sig + c, k);
}

// Eq. 1 numerators over one degree-bucket vertex list, G lanes per row (G = 4 for rows of
// at most 31 entries, G = 32 above): ACC = unsigned long long (integer weights, exact) or
// double.
template <typename ACC> __device__ __forceinline__ ACC acc_weight(const float *w, int64_t e);
template <> __device__ __forceinline__ unsigned long long acc_weight<unsigned long long>(const float *w, int64_t e)
{
    return w ? (unsigned long long)w[e] : 1ull;
}
template <> __device__ __forceinline__ double acc_weight<double>(const float *w, int64_t e)
{
    return w ? (double)w[e] : 1.0;
}

// Sums over entries e = start, start + STEP, ... < end of the row of vertex i (label ci):
// k += w_e, and in += w_e where the neighbour's label equals ci.  The graph is undirected with
// symmetric weights, so an edge {i, j} is counted from the entry with j > i at twice its weight
// (the entry j -> i holds the same weight) and a self-loop entry as it stands: half the label
// gathers, the same sums.  Four entries per round so that four label gathers are in flight
// per thread.
template <int STEP, typename ACC>
__device__ __forceinline__ void mod_row(const int32_t *idx, const float *w, const int32_t *C, int64_t start,
                                        int64_t end, int32_t i, int32_t ci, ACC &k, ACC &in)
{
    for (int64_t e = start; e < end; e += 4 * (int64_t)STEP) {
        int32_t j[4];
        ACC we[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t eu = e + (int64_t)u * STEP;
            j[u] = eu < end ? idx[eu] : -1;
            we[u] = eu < end ? acc_weight<ACC>(w, eu) : ACC(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            k += we[u];
            if (j[u] > i) {
                if (C[j[u]] == ci) in += we[u] + we[u];
            } else if (j[u] == i) {
                in += we[u];
            }
        }
    }
}

template <int G, typename ACC>
__global__ void __launch_bounds__(256) k_mod_list(const int64_t *off, const int32_t *idx, const float *w,
                                                  const int32_t *C, const int32_t *list, int64_t count, ACC *Sig,
                                                  ACC *acc)
{
    __shared__ int32_t sk[kModSlots];
    __shared__ ACC sv[kModSlots];
    __shared__ ACC s_in[8], s_k[8];
    for (int q = threadIdx.x; q < kModSlots; q += 256) {
        sk[q] = -1;
        sv[q] = ACC(0);
    }
    __syncthreads();
    const int lane = threadIdx.x & (G - 1);
    const unsigned gm = (G == 32) ? 0xFFFFFFFFu : (((1u << (G & 31)) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int64_t grp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / G;
    const int64_t ngrp = ((int64_t)gridDim.x * blockDim.x) / G;
    ACC tin = ACC(0), tk = ACC(0);
    for (int64_t r = grp; r < count; r += ngrp) {
        const int32_t i = list[r];
        const int64_t o0 = off[i], o1 = off[i + 1];
        const int32_t ci = C[i];
        ACC k = ACC(0), in = ACC(0);
        mod_row<G, ACC>(idx, w, C, o0 + lane, o1, i, ci, k, in);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            k += __shfl_xor_sync(gm, k, o);
            in += __shfl_xor_sync(gm, in, o);
        }
        if (lane == 0) {
            tin += in;
            tk += k;
            mod_sigma_add_t(sk, sv, Sig, ci, k);
        }
    }
    // block sums of sigma_in and 2m
#pragma unroll
    for (int o = 16; o >= G; o >>= 1) {
        tin += __shfl_xor_sync(0xFFFFFFFFu, tin, o);
        tk += __shfl_xor_sync(0xFFFFFFFFu, tk, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_in[threadIdx.x >> 5] = tin;
        s_k[threadIdx.x >> 5] = tk;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kModSlots; q += 256)
        if (sk[q] != -1) atomicAdd(Sig + sk[q], sv[q]);
    if (threadIdx.x == 0) {
        ACC a = ACC(0), b = ACC(0);
        for (int q = 0; q < 8; ++q) {
            a += s_in[q];
            b += s_k[q];
        }
        atomicAdd(acc + 0, a);
        atomicAdd(acc + 1, b);
    }
}

template <typename ACC>
__global__ void __launch_bounds__(256) k_mod_hub_chunks(const int32_t *idx, const float *w, const int32_t *C,
                                                        const int32_t *hub_v, const int32_t *chunk_h,
                                                        const int64_t *chunk_e0, const int64_t *chunk_e1, ACC *Sig,
                                                        ACC *acc)
{
    __shared__ ACC s_in[8], s_k[8];
    const int32_t v = hub_v[chunk_h[blockIdx.x]];
    const int32_t ci = C[v];
    ACC k = ACC(0), in = ACC(0);
    mod_row<256, ACC>(idx, w, C, chunk_e0[blockIdx.x] + threadIdx.x, chunk_e1[blockIdx.x], v, ci, k, in);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        k += __shfl_xor_sync(0xFFFFFFFFu, k, o);
        in += __shfl_xor_sync(0xFFFFFFFFu, in, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_in[threadIdx.x >> 5] = in;
        s_k[threadIdx.x >> 5] = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ACC a = ACC(0), b = ACC(0);
        for (int q = 0; q < 8; ++q) {
            a += s_in[q];
            b += s_k[q];
        }
        atomicAdd(acc + 0, a);
        atomicAdd(acc + 1, b);
        atomicAdd(Sig + ci, b);
    }
}

// Weight properties at creation: bit 1 of *flags is cleared when a weight is not an integer
// in [0, 2^24); *max_k receives the largest row sum (integer rows only).
__global__ void __launch_bounds__(256) k_weight_props(const int64_t *off, const float *w, int64_t n,
                                                      unsigned *flags, unsigned long long *max_k)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long mx = 0;
    bool integral = true;
    for (int64_t i = warp; i < n; i += nwarps) {
        unsigned long long k = 0;
        for (int64_t e = off[i] + lane; e < off[i + 1]; e += 32) {
            const float x = w ? w[e] : 1.0f;
            if (!(x >= 0.0f && x < 16777216.0f && truncf(x) == x)) integral = false;
            k += (unsigned long long)x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xFFFFFFFFu, k, o);
        mx = k > mx ? k : mx;
    }
    if (!integral) atomicAnd(flags, ~2u);
    if (lane == 0 && mx) atomicMax(max_k, mx);
}

// Flat pass over all weights: bit 1 of *flags is cleared when a weight is not an integer in
// [0, 2^24), bit 2 when a weight is not exactly 1; *wmax_bits receives the bits of the
// largest weight (non-negative floats order like their bit patterns).  Row sums are needed
// only when max weight x max degree can reach 2^24 (then k_weight_props computes them).
__global__ void __launch_bounds__(256) k_weight_flat(const float *w, int64_t m, unsigned *flags, unsigned *wmax_bits)
{
    bool integral = true, ones = true;
    float mx = 0.0f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const float x = w[e];
        if (!(x >= 0.0f && x < 16777216.0f && truncf(x) == x)) integral = false;
        if (x != 1.0f) ones = false;
        mx = fmaxf(mx, x);
    }
    integral = __all_sync(0xFFFFFFFFu, integral);
    ones = __all_sync(0xFFFFFFFFu, ones);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if ((threadIdx.x & 31) == 0) {
        if (!integral) atomicAnd(flags, ~2u);
        if (!ones) atomicAnd(flags, ~4u);
        atomicMax(wmax_bits, __float_as_uint(mx));
    }
}

__global__ void __launch_bounds__(256) k_degree_max(const int64_t *off, int64_t n, unsigned long long *dmax)
{
    unsigned long long mx = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long d = (unsigned long long)(off[i + 1] - off[i]);
        mx = d > mx ? d : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, mx, o);
        mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(dmax, mx);
}

// Integer-weight modularity: every sum is an exact integer (int64 for sigma, Sigma_c and 2m,
// 128 bits for sum_c Sigma_c^2), so Q is exact up to the final division and independent of
// the order of the atomics.
// Integer weights: every sum is an exact integer (int64 for sigma, Sigma_c and 2m, 128 bits
// for sum_c Sigma_c^2), so Q is exact up to the final division and independent of the
// order of the atomics.  sum_c Sigma_c^2 goes to acc[2] (low word) and acc[3] (high word);
// Sigma is reset for the next call.
__device__ __forceinline__ void add128(unsigned long long &lo, unsigned long long &hi, unsigned long long xl,
                                       unsigned long long xh)
{
    const unsigned long long r = lo + xl;
    hi += xh + (r < lo ? 1ull : 0ull);
    lo = r;
}

__global__ void __launch_bounds__(256) k_mod_sq_int(unsigned long long *Sig, int64_t n, unsigned long long *acc)
{
    __shared__ unsigned long long s_lo[8], s_hi[8];
    unsigned long long lo = 0, hi = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long x = Sig[c];
        if (x) {
            add128(lo, hi, x * x, __umul64hi(x, x));
            Sig[c] = 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        add128(lo, hi, __shfl_xor_sync(0xFFFFFFFFu, lo, o), __shfl_xor_sync(0xFFFFFFFFu, hi, o));
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        lo = 0;
        hi = 0;
        for (int q = 0; q < 8; ++q) add128(lo, hi, s_lo[q], s_hi[q]);
        const unsigned long long old = atomicAdd(acc + 2, lo);
        atomicAdd(acc + 3, hi + (old + lo < old ? 1ull : 0ull));
    }
}

__global__ void __launch_bounds__(256) k_mod_sq(double *Sig, int64_t n, double *acc)
{
    __shared__ double s[8];
    double t = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const double x = Sig[c];
        if (x != 0.0) {
            t += x * x;
            Sig[c] = 0.0;
        }
    }
    t = warp_sum_d(t);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < 8; ++q) a += s[q];
        atomicAdd(acc + 2, a);
    }
}

int grid_for(int64_t work, int threads, int max_per_sm = 8)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int64_t b = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)sms * max_per_sm;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

uint32_t capacity_bits(int64_t x)
{
    uint32_t b = 1;
    while (b < 31 && ((int64_t)1 << b) - 1 < x) ++b;
    return b;
}

}  // namespace
// ---------------------------------------------------------------------------------------
// Device memory arena

namespace lpa {

Arena::Arena(size_t bytes, bool grow, size_t grow_chunk) : grow_(grow), grow_chunk_(grow_chunk)
{
    if (bytes > 0) add_region(bytes);
}

Arena::~Arena()
{
    for (Region &r : regions_)
        if (r.base) cudaFree(r.base);
}

bool Arena::add_region(size_t bytes)
{
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    Region r;
    r.base = static_cast<unsigned char *>(p);
    r.cap = bytes;
    r.free_.emplace(0, bytes);
    regions_.push_back(std::move(r));
    return true;
}

// First fit in offset order; ordered maps keep allocation and release logarithmic, so that a
// batch of thousands of graphs (tens of thousands of blocks) is created and released quickly.
void *Arena::region_alloc(Region &r, size_t bytes)
{
    for (auto it = r.free_.begin(); it != r.free_.end(); ++it) {
        if (it->second < bytes) continue;
        const size_t off = it->first, size = it->second;
        r.free_.erase(it);
        if (size > bytes) r.free_.emplace(off + bytes, size - bytes);
        r.taken_.emplace(off, bytes);
        r.used += bytes;
        return r.base + off;
    }
    return nullptr;
}

void *Arena::alloc(size_t bytes)
{
    std::lock_guard<std::mutex> lock(mu_);
    bytes = (std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
    for (Region &r : regions_)
        if (void *p = region_alloc(r, bytes)) return p;
    if (!grow_ || !add_region(std::max(bytes, grow_chunk_))) return nullptr;
    return region_alloc(regions_.back(), bytes);
}

void Arena::free(void *p)
{
    if (!p) return;
    std::lock_guard<std::mutex> lock(mu_);
    unsigned char *q = static_cast<unsigned char *>(p);
    for (Region &r : regions_) {
        if (q < r.base || q >= r.base + r.cap) continue;
        const size_t off = (size_t)(q - r.base);
        auto t = r.taken_.find(off);
        if (t == r.taken_.end()) return;
        size_t start = off, size = t->second;
        r.taken_.erase(t);
        r.used -= size;
        auto next = r.free_.lower_bound(start);
        if (next != r.free_.end() && start + size == next->first) {   // merge with the next block
            size += next->second;
            next = r.free_.erase(next);
        }
        if (next != r.free_.begin()) {                                  // and with the previous one
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                size += prev->second;
                r.free_.erase(prev);
            }
        }
        r.free_.emplace(start, size);
        return;
    }
}

size_t Arena::capacity() const
{
    size_t c = 0;
    for (const Region &r : regions_) c += r.cap;
    return c;
}

size_t Arena::used() const
{
    size_t u = 0;
    for (const Region &r : regions_) u += r.used;
    return u;
}

size_t Arena::largest_free() const
{
    size_t m = 0;
    for (const Region &r : regions_)
        for (const auto &b : r.free_) m = std::max(m, b.second);
    return m;
}

}  // namespace lpa

// ---------------------------------------------------------------------------------------
namespace {

// Host-side fault injection (lpa_debug_fail_allocations): the number of further device
// allocations that succeed before every later one fails; negative = off.
std::atomic<long long> g_alloc_budget{-1};

bool injected_alloc_failure()
{
    long long b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) return true;
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) return false;
    }
    return false;
}

// Device memory of single-graph handles comes from a stream-ordered pool per device that keeps
// freed blocks (release threshold: never), so creating a handle after destroying another does
// not pay for cudaMalloc / cudaFree of gigabytes again; lpa_trim_memory returns the cached
// blocks to the driver.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxPoolDevices] = {};

cudaMemPool_t handle_pool(int dev)
{
    if (dev < 0 || dev >= kMaxPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}

template <typename T>
int dalloc(lpa_graph *g, T **p, size_t count)
{
    *p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    void *q = nullptr;
    if (injected_alloc_failure()) {
        set_error("device allocation of " + std::to_string(bytes) + " bytes failed (injected)");
        return LPA_ENOMEM;
    }
    if (g->arena) {
        q = g->arena->alloc(bytes);
    } else {
        cudaMemPool_t pool = handle_pool(g->device);
        const cudaError_t e = pool ? cudaMallocFromPoolAsync(&q, bytes, pool, g->stream) : cudaMalloc(&q, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            q = nullptr;
        }
    }
    if (!q) {
        set_error("device allocation of " + std::to_string(bytes) + " bytes failed" +
                  (g->arena ? " (arena full)" : ""));
        return LPA_ENOMEM;
    }
    g->allocs.push_back({q, bytes});
    g->bytes += (int64_t)bytes;
    *p = static_cast<T *>(q);
    return LPA_OK;
}

void dfree(lpa_graph *g, void *p)
{
    if (!p) return;
    for (size_t i = 0; i < g->allocs.size(); ++i) {
        if (g->allocs[i].first != p) continue;
        g->bytes -= (int64_t)g->allocs[i].second;
        g->allocs.erase(g->allocs.begin() + (long)i);
        break;
    }
    if (g->arena) g->arena->free(p);
    else cudaFreeAsync(p, g->stream);
}

lpa_tuning default_tuning()
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
    t.item_vertices = 0;
    t.hub_chunk = 16384;
    t.hub_table_shift = 1;
    t.smem_table_shift = 1;
    t.probe = 4;                                      // quadratic-double over power-of-two tables
    t.flat_buckets = 0;                               // one thread / lane group / warp per vertex
    t.hub_two_pass = 1;                               // hubs in two passes in a run's first sweep
    return t;
}

// smem slots of a bucket whose largest degree is dmax: capacity(dmax << shift) + 1
int64_t slots_for(int64_t dmax, int shift)
{
    return (int64_t)1 << capacity_bits(std::max<int64_t>(dmax, 1) << shift);
}

int check_tuning(const lpa_tuning &t)
{
    auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
    if (t.smem_table_shift < 0 || t.smem_table_shift > 2) return LPA_EINVAL;
    if (t.hub_table_shift < 0 || t.hub_table_shift > 3) return LPA_EINVAL;
    const int sh = t.smem_table_shift;
    if (t.thread_max < 0 || slots_for(t.thread_max, sh) > 16) return LPA_EINVAL;
    if (t.group_max < t.thread_max || t.warp_max < t.group_max || t.cta_max < t.warp_max ||
        t.cta_large_max < t.cta_max || t.cta_xl_max < t.cta_large_max)
        return LPA_EINVAL;
    if (!(t.group_lanes == 2 || t.group_lanes == 4 || t.group_lanes == 8 || t.group_lanes == 16)) return LPA_EINVAL;
    for (int th : {t.cta_threads, t.cta_large_threads, t.cta_xl_threads})
        if (!pow2(th) || th < 64 || th > 1024) return LPA_EINVAL;
    if (t.hub_chunk < 256 || t.hub_chunk > 32768) return LPA_EINVAL;
    if (t.item_vertices < 0 || t.item_vertices > (1 << 20)) return LPA_EINVAL;
    if (t.float_values < 0 || t.float_values > 2) return LPA_EINVAL;
    if (t.hub_cluster != 0 && t.hub_cluster != 1) return LPA_EINVAL;
    if (t.probe < 0 || t.probe > 4) return LPA_EINVAL;
    if (t.flat_buckets < 0 || t.flat_buckets > 7) return LPA_EINVAL;
    if (t.hub_two_pass < 0 || t.hub_two_pass > 2) return LPA_EINVAL;
    for (int r : t.reserved)
        if (r != 0) return LPA_EINVAL;
    const int64_t smem = (int64_t)max_dynamic_smem();
    const int64_t sb = t.float_values == 2 ? 12 : 8;  // bytes per slot: key + value
    const int64_t bytes_group = (256 / t.group_lanes) * slots_for(t.group_max, sh) * sb;
    const int64_t bytes_warp = 8 * slots_for(t.warp_max, sh) * sb;
    const int64_t bytes_cta = slots_for(t.cta_max, sh) * sb;
    const int64_t bytes_large = slots_for(t.cta_large_max, sh) * sb;
    const int64_t bytes_xl = slots_for(t.cta_xl_max, sh) * sb;
    if (bytes_group > smem || bytes_warp > smem || bytes_cta > smem || bytes_large > smem || bytes_xl > smem)
        return LPA_EINVAL;
    return LPA_OK;
}

// Vertices per work item of each vertex kernel (a warp's or a block's unit of queue work).
int64_t item_size(const lpa_tuning &t, int b)
{
    static const int64_t base[B_CTA_XL + 1] = {1024, 256, 64, 16, 8, 4};
    if (t.item_vertices > 0 && b <= B_WARP) return t.item_vertices;
    return base[b];
}

void free_buckets(lpa_graph *g)
{
    dfree(g, g->lists);
    g->lists = nullptr;
    dfree(g, g->hub_mem);
    g->hub_mem = nullptr;
    dfree(g, g->tab_k);                               // tab_v lives in the same block
    g->tab_k = nullptr;
    g->tab_v = nullptr;
    dfree(g, g->used_list);
    g->used_list = nullptr;
    dfree(g, g->pairs);
    g->pairs = nullptr;
    dfree(g, g->items_d);
    g->items_d = nullptr;
    g->gdh.hub = HubArgs{};
    g->table_slots = 0;
    for (auto &v : g->items_h) v.clear();
    for (auto &v : g->hub_items_h) v.clear();
}

int build_buckets(lpa_graph *g)
{
    free_buckets(g);
    const int64_t n = g->n;
    const int64_t tiles = (n + 1023) / 1024;
    std::vector<int32_t> cnt((size_t)std::max<int64_t>(tiles, 1) * B_COUNT, 0);
    std::vector<int64_t> base(cnt.size(), 0);
    int32_t *d_cnt = nullptr;
    int64_t *d_base = nullptr;
    LPA_CHECK(dalloc(g, &d_cnt, cnt.size()));
    int st = dalloc(g, &d_base, base.size());
    if (st != LPA_OK) {
        dfree(g, d_cnt);
        return st;
    }
    auto cleanup = [&]() {
        dfree(g, d_cnt);
        dfree(g, d_base);
    };
    if (tiles > 0) {
        k_bucket_count<<<(unsigned)tiles, 1024, 0, g->stream>>>(g->off, n, g->tuning, d_cnt);
        cudaMemcpyAsync(cnt.data(), d_cnt, cnt.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream);
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) {
            cleanup();
            set_error(std::string("bucket count: ") + cudaGetErrorString(e));
            return LPA_ECUDA;
        }
    }
    int64_t total[B_COUNT] = {};
    for (int64_t t = 0; t < tiles; ++t)
        for (int b = 0; b < B_COUNT; ++b) total[b] += cnt[t * B_COUNT + b];
    g->bucket_start[0] = 0;
    for (int b = 0; b < B_COUNT; ++b) g->bucket_start[b + 1] = g->bucket_start[b] + total[b];
    int64_t run[B_COUNT];
    for (int b = 0; b < B_COUNT; ++b) run[b] = g->bucket_start[b];
    for (int64_t t = 0; t < tiles; ++t)
        for (int b = 0; b < B_COUNT; ++b) {
            base[t * B_COUNT + b] = run[b];
            run[b] += cnt[t * B_COUNT + b];
        }
    st = dalloc(g, &g->lists, (size_t)g->bucket_start[B_COUNT]);
    if (st != LPA_OK) {
        cleanup();
        return st;
    }
    if (tiles > 0) {
        cudaMemcpyAsync(d_base, base.data(), base.size() * sizeof(int64_t), cudaMemcpyHostToDevice, g->stream);
        k_bucket_fill<<<(unsigned)tiles, 1024, 0, g->stream>>>(g->off, n, g->tuning, d_base, g->lists);
    }
    cudaError_t e = cudaStreamSynchronize(g->stream);
    cleanup();
    if (e != cudaSuccess) {
        set_error(std::string("bucket fill: ") + cudaGetErrorString(e));
        return LPA_ECUDA;
    }

    // vertex work items
    const int64_t *bs = g->bucket_start;
    for (int b = B_THREAD; b <= B_CTA_XL; ++b) {
        const int64_t sz = item_size(g->tuning, b);
        for (int64_t s = bs[b]; s < bs[b + 1]; s += sz)
            g->items_h[b].push_back(WorkItem{0, 0, s, std::min(sz, bs[b + 1] - s)});
    }

    // hubs: tables in HBM, accumulate chunks and clear slices
    HubArgs &ha = g->gdh.hub;
    const int64_t H = total[B_HUB];
    if (H > 0) {
        const int32_t *hub_list = g->lists + bs[B_HUB];
        std::vector<int32_t> hv((size_t)H);
        std::vector<int64_t> o0((size_t)H), o1((size_t)H);
        int64_t *d_o = nullptr;
        LPA_CHECK(dalloc(g, &d_o, (size_t)(2 * H)));
        k_gather_rows<<<(unsigned)((H + 255) / 256), 256, 0, g->stream>>>(hub_list, H, g->off, d_o, d_o + H);
        cudaMemcpyAsync(hv.data(), hub_list, H * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream);
        cudaMemcpyAsync(o0.data(), d_o, H * sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream);
        cudaMemcpyAsync(o1.data(), d_o + H, H * sizeof(int64_t), cudaMemcpyDeviceToHost, g->stream);
        e = cudaStreamSynchronize(g->stream);
        dfree(g, d_o);
        if (e != cudaSuccess) {
            set_error(std::string("hub rows: ") + cudaGetErrorString(e));
            return LPA_ECUDA;
        }
        const int64_t chunk = g->tuning.hub_chunk;
        std::vector<uint32_t> p1((size_t)H), bb((size_t)H);
        std::vector<int64_t> tab((size_t)H), ubase((size_t)H);
        std::vector<int32_t> ch, sh, sj;
        std::vector<int64_t> ce0, ce1;
        int64_t slots = 0, used_total = 0;
        // With hub_cluster, tables of at most 2^kDsmMaxBits slots (integer sums) live in the
        // shared memory of a cluster of 2..16 blocks; the others live in HBM with accumulate
        // chunks and clear slices.
        const int dsm_bits = (g->tuning.hub_cluster && plan_int_weights(g)) ? dsm_max_class_bits() : 0;
        const bool dsm_ok = dsm_bits > 0;
        std::vector<int64_t> acc_chunks;
        // two-pass accumulation for integer sums with HBM tables: first-pass chunks and partitions
        const bool two_pass = plan_int_weights(g) && g->tuning.hub_two_pass;
        std::vector<uint32_t> hpb((size_t)H, 0u);
        std::vector<int32_t> hpbase((size_t)H, -1), pch, parth;
        std::vector<int64_t> pce0, pce1;
        for (int64_t h = 0; h < H; ++h) {
            const int64_t D = o1[h] - o0[h];
            // capacity_bits stops at 31: p1 <= 2^31 - 1 still holds every distinct label (labels
            // are below n < 2^31), the probe's secondary modulus 2 p1 + 1 fits in 32 bits and
            // the remainder multipliers are indexed at b + 1 <= 32, inside their table.
            const int64_t want = std::min<int64_t>(D << g->tuning.hub_table_shift, (int64_t)1 << 31);
            bb[h] = capacity_bits(want);
            p1[h] = (uint32_t)(((int64_t)1 << bb[h]) - 1);
            const bool dsm = dsm_ok && (int)bb[h] <= kDsmSliceBits + dsm_bits;
            for (int64_t e0 = o0[h]; e0 < o1[h]; e0 += chunk) {
                ch.push_back((int32_t)h);
                ce0.push_back(e0);
                ce1.push_back(std::min(o1[h], e0 + chunk));
            }
            if (dsm) {
                const int cs_bits = std::min(4, std::max(1, (int)bb[h] - kDsmSliceBits));
                g->hub_items_h[HL_DSM2 + cs_bits - 1].push_back(WorkItem{0, 0, h, 1});
                tab[h] = -1;
                ubase[h] = -1;
                continue;
            }
            if (two_pass) {
                uint32_t pb = 0;
                while (pb < (uint32_t)kPartMaxBits && ((D + ((int64_t)1 << pb) - 1) >> pb) > kPartExpect) ++pb;
                hpb[h] = pb;
                hpbase[h] = (int32_t)parth.size();
                for (uint32_t q = 0; q < (1u << pb); ++q) parth.push_back((int32_t)h);
                for (int64_t e0 = o0[h]; e0 < o1[h]; e0 += kPartChunk) {
                    pch.push_back((int32_t)h);
                    pce0.push_back(e0);
                    pce1.push_back(std::min<int64_t>(o1[h], e0 + kPartChunk));
                }
            }
            if (!two_pass || g->tuning.hub_two_pass == 1) {     // single-pass accumulate chunks
                for (int64_t c = (int64_t)ch.size() - (o1[h] - o0[h] + chunk - 1) / chunk; c < (int64_t)ch.size(); ++c)
                    acc_chunks.push_back(c);
            }
            tab[h] = slots;
            ubase[h] = used_total;
            // 2^b = p1 + 1 slots: Algorithm 2 probes p1 of them, the power-of-two probe all
            for (int64_t j = 0; j * kHubSlice < (int64_t)p1[h] + 1; ++j) {   // clear slices cover the table
                sh.push_back((int32_t)h);
                sj.push_back((int32_t)j);
            }
            slots += (int64_t)p1[h] + 1;
            used_total += D;
        }
        const int64_t n_chunks = (int64_t)ch.size(), n_slices = (int64_t)sh.size();
        g->table_slots = slots;
        const bool f64 = g->tuning.float_values == 2;   // float64 values: per-chunk arg-max pairs
        const int64_t n_pch = (int64_t)pch.size(), n_parts = (int64_t)parth.size();
        const size_t n8 = (size_t)(3 * H + 2 * n_chunks + (f64 ? n_chunks : 0) + 2 * n_pch);
        const size_t n4 = (size_t)(4 * H + n_chunks + 2 * n_slices + (f64 ? n_chunks + H + 1 : 0) + n_pch + 2 * H +
                                   3 * n_parts);
        unsigned char *mem = nullptr;
        LPA_CHECK(dalloc(g, &mem, n8 * 8 + n4 * 4 + 2 * (size_t)H));
        g->hub_mem = mem;
        unsigned char *p = mem;
        auto take = [&](size_t b) {
            unsigned char *r = p;
            p += b;
            return r;
        };
        int64_t *d_tab = (int64_t *)take(H * 8);
        unsigned long long *d_best = (unsigned long long *)take(H * 8);
        int64_t *d_ubase = (int64_t *)take(H * 8);
        int64_t *d_ce0 = (int64_t *)take(n_chunks * 8);
        int64_t *d_ce1 = (int64_t *)take(n_chunks * 8);
        double *d_cbv = f64 ? (double *)take(n_chunks * 8) : nullptr;
        int64_t *d_pce0 = (int64_t *)take(n_pch * 8);
        int64_t *d_pce1 = (int64_t *)take(n_pch * 8);
        int32_t *d_hv = (int32_t *)take(H * 4);
        uint32_t *d_p1 = (uint32_t *)take(H * 4);
        uint32_t *d_b = (uint32_t *)take(H * 4);
        uint32_t *d_used = (uint32_t *)take(H * 4);
        int32_t *d_ch = (int32_t *)take(n_chunks * 4);
        int32_t *d_sh = (int32_t *)take(n_slices * 4);
        int32_t *d_sj = (int32_t *)take(n_slices * 4);
        int32_t *d_cbk = f64 ? (int32_t *)take(n_chunks * 4) : nullptr;
        int32_t *d_hc0 = f64 ? (int32_t *)take((H + 1) * 4) : nullptr;
        int32_t *d_pch = (int32_t *)take(n_pch * 4);
        uint32_t *d_hpb = (uint32_t *)take(H * 4);
        int32_t *d_hpbase = (int32_t *)take(H * 4);
        int32_t *d_parth = (int32_t *)take(n_parts * 4);
        uint32_t *d_pcnt = (uint32_t *)take(n_parts * 4);
        int32_t *d_povf = (int32_t *)take(n_parts * 4);
        uint8_t *d_act = (uint8_t *)take(H);
        uint8_t *d_seen = (uint8_t *)take(H);
        LPA_CUDA(cudaMemcpyAsync(d_tab, tab.data(), H * 8, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_ubase, ubase.data(), H * 8, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_ce0, ce0.data(), n_chunks * 8, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_ce1, ce1.data(), n_chunks * 8, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_hv, hv.data(), H * 4, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_p1, p1.data(), H * 4, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_b, bb.data(), H * 4, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_ch, ch.data(), n_chunks * 4, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_sh, sh.data(), n_slices * 4, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_sj, sj.data(), n_slices * 4, cudaMemcpyHostToDevice, g->stream));
        if (n_pch > 0) {
            LPA_CUDA(cudaMemcpyAsync(d_pce0, pce0.data(), n_pch * 8, cudaMemcpyHostToDevice, g->stream));
            LPA_CUDA(cudaMemcpyAsync(d_pce1, pce1.data(), n_pch * 8, cudaMemcpyHostToDevice, g->stream));
            LPA_CUDA(cudaMemcpyAsync(d_pch, pch.data(), n_pch * 4, cudaMemcpyHostToDevice, g->stream));
        }
        LPA_CUDA(cudaMemcpyAsync(d_hpb, hpb.data(), H * 4, cudaMemcpyHostToDevice, g->stream));
        LPA_CUDA(cudaMemcpyAsync(d_hpbase, hpbase.data(), H * 4, cudaMemcpyHostToDevice, g->stream));
        if (n_parts > 0) {
            LPA_CUDA(cudaMemcpyAsync(d_parth, parth.data(), n_parts * 4, cudaMemcpyHostToDevice, g->stream));
            LPA_CUDA(cudaMemsetAsync(d_pcnt, 0, n_parts * 8, g->stream));       // part_cnt and part_ovf
            LPA_CHECK(dalloc(g, &g->pairs, (size_t)n_parts * kPartCap));
        }
        LPA_CUDA(cudaMemsetAsync(d_act, 0, 2 * H, g->stream));     // hub_act and hub_seen
        LPA_CUDA(cudaMemsetAsync(d_best, 0, H * 8, g->stream));
        LPA_CUDA(cudaMemsetAsync(d_used, 0, H * 4, g->stream));
        if (f64) {
            std::vector<int32_t> hc0((size_t)H + 1, (int32_t)n_chunks);
            for (int64_t c = n_chunks - 1; c >= 0; --c) hc0[(size_t)ch[(size_t)c]] = (int32_t)c;
            LPA_CUDA(cudaMemcpyAsync(d_hc0, hc0.data(), (H + 1) * 4, cudaMemcpyHostToDevice, g->stream));
            LPA_CUDA(cudaStreamSynchronize(g->stream));
        }
        // 8 bytes per slot in one block: split keys then values, or packed 64-bit slots; with
        // float64 values 12 bytes: keys, then the values from an 8-byte boundary
        const int64_t keys_even = (std::max<int64_t>(slots, 2) + 1) & ~(int64_t)1;
        LPA_CHECK(dalloc(g, &g->tab_k, (size_t)(f64 ? 3 * keys_even : std::max<int64_t>(slots, 2) * 2)));
        g->tab_v = reinterpret_cast<float *>(g->tab_k + slots);                       // (none when every hub
        double *tab_vd = f64 ? reinterpret_cast<double *>(g->tab_k + keys_even) : nullptr;   //  is in a cluster)
        LPA_CHECK(dalloc(g, &g->used_list, (size_t)std::max<int64_t>(used_total, 1)));
        LPA_CUDA(launch_hub_table_clear(g->tab_k, g->tab_v, slots, plan_int_weights(g), g->stream, tab_vd));
        ha.hub_v = d_hv;
        ha.hub_p1 = d_p1;
        ha.hub_b = d_b;
        ha.hub_tab = d_tab;
        ha.hub_act = d_act;
        ha.hub_seen = d_seen;
        ha.hub_best = d_best;
        ha.hub_used = d_used;
        ha.used_list = g->used_list;
        ha.used_base = d_ubase;
        ha.chunk_h = d_ch;
        ha.chunk_e0 = d_ce0;
        ha.chunk_e1 = d_ce1;
        ha.slice_h = d_sh;
        ha.slice_j = d_sj;
        ha.tab_k = g->tab_k;
        ha.tab_v = g->tab_v;
        ha.tab_vd = tab_vd;
        ha.chunk_bv = d_cbv;
        ha.chunk_bk = d_cbk;
        ha.hub_c0 = d_hc0;
        ha.pc_h = d_pch;
        ha.pc_e0 = d_pce0;
        ha.pc_e1 = d_pce1;
        ha.hub_pb = d_hpb;
        ha.hub_pbase = d_hpbase;
        ha.part_h = d_parth;
        ha.part_cnt = d_pcnt;
        ha.part_ovf = d_povf;
        ha.pairs = g->pairs;
        ha.n_hubs = (int32_t)H;
        ha.n_chunks = (int32_t)n_chunks;
        ha.n_slices = (int32_t)n_slices;
        for (int64_t h0 = 0; h0 < H; h0 += 256)
            g->hub_items_h[HL_HUBS].push_back(WorkItem{0, 0, h0, std::min<int64_t>(256, H - h0)});
        for (int64_t c : acc_chunks) g->hub_items_h[HL_ACC].push_back(WorkItem{0, 0, c, 1});
        for (int64_t c = 0; c < n_chunks; ++c) g->hub_items_h[HL_MARK].push_back(WorkItem{0, 0, c, 1});
        for (int64_t j = 0; j < n_slices; ++j) g->hub_items_h[HL_SLICES].push_back(WorkItem{0, 0, j, 1});
        for (int64_t c = 0; c < n_pch; ++c) g->hub_items_h[HL_PACC].push_back(WorkItem{0, 0, c, 1});
        for (int64_t q = 0; q < n_parts; ++q) g->hub_items_h[HL_PMERGE].push_back(WorkItem{0, 0, q, 1});
    }

    // every item of this graph in one device block: vertex items, hub items, one per-graph item
    size_t total_items = 1;
    for (int b = B_THREAD; b <= B_CTA_XL; ++b) total_items += g->items_h[b].size();
    for (int q = 0; q < HL_COUNT; ++q) total_items += g->hub_items_h[q].size();
    std::vector<WorkItem> all;
    all.reserve(total_items);
    size_t at[B_COUNT] = {}, at_h[HL_COUNT] = {}, at_pg = 0;
    for (int b = B_THREAD; b <= B_CTA_XL; ++b) {
        at[b] = all.size();
        all.insert(all.end(), g->items_h[b].begin(), g->items_h[b].end());
    }
    for (int q = 0; q < HL_COUNT; ++q) {
        at_h[q] = all.size();
        all.insert(all.end(), g->hub_items_h[q].begin(), g->hub_items_h[q].end());
    }
    at_pg = all.size();
    all.push_back(WorkItem{0, 0, 0, 0});
    LPA_CHECK(dalloc(g, &g->items_d, all.size()));
    LPA_CUDA(cudaMemcpyAsync(g->items_d, all.data(), all.size() * sizeof(WorkItem), cudaMemcpyHostToDevice,
                             g->stream));
    for (int b = B_THREAD; b <= B_CTA_XL; ++b) g->items_at[b] = g->items_d + at[b];
    for (int q = 0; q < HL_COUNT; ++q) g->hub_items_d[q] = g->items_d + at_h[q];
    g->per_graph_d = g->items_d + at_pg;
    LPA_CHECK(upload_descriptor(g));
    LPA_CUDA(cudaStreamSynchronize(g->stream));
    return LPA_OK;
}

cudaEvent_t event_at(lpa_graph *g, size_t k)
{
    while (g->events.size() <= k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        g->events.push_back(e);
    }
    return g->events[k];
}

int init_state(lpa_graph *g)
{
    if (g->n > 0) {
        k_init_labels<<<grid_for(g->n, 256, 16), 256, 0, g->stream>>>(g->off, g->n, g->C, g->flags[0]);
        LPA_CUDA(cudaGetLastError());
        LPA_CUDA(cudaMemsetAsync(g->flags[1], 0, (size_t)g->n, g->stream));
    }
    g->active_buf = 0;
    g->next_iter = 0;
    return LPA_OK;
}

// CUDA-event timing of every launch of lpa_run (stats->time_kernels).
struct EventHook : LaunchHook {
    lpa_graph *g;
    size_t *evn;
    int iter = 0;
    bool on = false;
    struct Rec {
        int iter, slot;
        size_t e0, e1;
    };
    std::vector<Rec> recs;
    size_t pending = 0;
    EventHook(lpa_graph *gg, size_t *n) : g(gg), evn(n) {}
    void before(int slot) override
    {
        (void)slot;
        if (!on) return;
        pending = (*evn)++;
        cudaEvent_t e = event_at(g, pending);
        if (e) cudaEventRecord(e, g->stream);
    }
    void after(int slot) override
    {
        if (!on) return;
        const size_t e1 = (*evn)++;
        cudaEvent_t e = event_at(g, e1);
        if (e) cudaEventRecord(e, g->stream);
        recs.push_back({iter, slot, pending, e1});
    }
};

}  // namespace

// ---------------------------------------------------------------------------------------
namespace lpa {

int ensure_counters(lpa_graph *g, int iters, bool mirror)
{
    if (iters < 1) iters = 1;
    if (iters > g->ctr_iters) {
        dfree(g, g->ctr);
        g->ctr = nullptr;
        g->ctr_iters = 0;
        LPA_CHECK(dalloc(g, &g->ctr, (size_t)kPerSweep * iters));
        g->ctr_iters = iters;
    }
    if (mirror && iters > g->h_ctr_iters) {
        if (g->h_ctr) cudaFreeHost(g->h_ctr);
        g->h_ctr = nullptr;
        g->h_ctr_iters = 0;
        if (cudaMallocHost((void **)&g->h_ctr, (size_t)kPerSweep * iters * sizeof(unsigned long long)) !=
            cudaSuccess) {
            cudaGetLastError();
            g->h_ctr = nullptr;
            set_error("cudaMallocHost failed");
            return LPA_ENOMEM;
        }
        g->h_ctr_iters = iters;
    }
    return LPA_OK;
}

void plan_slots(const lpa_tuning &t, int32_t slots[B_COUNT])
{
    const int sh = t.smem_table_shift;
    slots[B_THREAD] = 16;
    slots[B_GROUP] = (int32_t)slots_for(t.group_max, sh);
    slots[B_WARP] = (int32_t)slots_for(t.warp_max, sh);
    slots[B_CTA] = (int32_t)slots_for(t.cta_max, sh);
    slots[B_CTA_LARGE] = (int32_t)slots_for(t.cta_large_max, sh);
    slots[B_CTA_XL] = (int32_t)slots_for(t.cta_xl_max, sh);
    slots[B_HUB] = 0;
}

bool plan_int_weights(const lpa_graph *g) { return g->int_weights && !g->tuning.float_values; }

int upload_descriptor(lpa_graph *g)
{
    GraphDev &d = g->gdh;
    d.off = g->off;
    d.idx = g->idx;
    d.w = g->w;
    d.C = g->C;
    d.flags0 = g->flags[0];
    d.flags1 = g->flags[1];
    d.mover_v = g->mover_v;
    d.mover_v1 = g->mover_v1;
    d.cc_prev = g->cc_prev;
    d.cc_midx = g->cc_midx;
    d.cc_par0 = g->cc_par0;
    d.cc_word = g->cc_word;
    d.mover_c = g->mover_c;
    d.mover_count = g->mover_count;
    d.ctr = g->ctr;
    d.ctr_iters = g->ctr_iters;
    d.fallbacks = g->fallbacks;
    d.lists = g->lists;
    d.rs = g->rs_d;
    d.tshift = g->tuning.smem_table_shift;
    d.probe = g->tuning.probe;
    d.int_weights = plan_int_weights(g) ? 1 : 0;
    d.hub_tp = plan_int_weights(g) ? g->tuning.hub_two_pass : 0;     // the lists exist for integer sums
    d.hub_deg = g->tuning.cta_xl_max;
    d.rows_strict = g->rows_strict ? 1 : 0;
    LPA_CUDA(cudaMemcpyAsync(g->gdd, &g->gdh, sizeof(GraphDev), cudaMemcpyHostToDevice, g->stream));
    return LPA_OK;
}

void destroy_graph(lpa_graph *g, bool arena_released)
{
    if (!g) return;
    DeviceGuard dg(g->device);
    if (arena_released && g->arena) {                 // the owner releases the whole arena after this
        g->allocs.clear();
    } else if (g->stream) {
        cudaStreamSynchronize(g->stream);
    }
    for (auto &a : g->allocs) {
        if (g->arena) g->arena->free(a.first);
        else cudaFreeAsync(a.first, g->stream);
    }
    g->allocs.clear();
    if (g->stream && !g->arena) cudaStreamSynchronize(g->stream);
    if (g->h_ctr) cudaFreeHost(g->h_ctr);
    if (g->hm) cudaFreeHost(g->hm);
    for (cudaEvent_t e : g->events) cudaEventDestroy(e);
    delete g;
}

int create_graph(const void *offsets, const int32_t *indices, const float *weights, int64_t n_vertices,
                 int64_t n_entries, int flags, cudaStream_t stream, Arena *arena, const lpa_tuning *tuning,
                 lpa_graph **out)
{
    if (!out) {
        set_error("lpa_create: out is NULL");
        return LPA_EINVAL;
    }
    *out = nullptr;
    if (n_vertices < 0 || n_vertices >= ((int64_t)1 << 31) - 1 || n_entries < 0 || !offsets ||
        (n_entries > 0 && !indices)) {
        set_error("lpa_create: bad sizes or NULL arrays");
        return LPA_EINVAL;
    }
    if ((flags & LPA_OFFSETS_I64) == 0 && n_entries > INT32_MAX) {
        set_error("lpa_create: int32 offsets cannot address more than 2^31-1 entries");
        return LPA_EINVAL;
    }
    lpa_graph *g = new lpa_graph();
    cudaGetDevice(&g->device);
    g->stream = stream;
    g->arena = arena;
    g->n = n_vertices;
    g->m = n_entries;
    g->tuning = tuning ? *tuning : default_tuning();
    const bool dev_ptrs = (flags & LPA_DEVICE_PTRS) != 0;
    const cudaMemcpyKind kind = dev_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    int st = LPA_OK;
    auto fail = [&](int s) {
        destroy_graph(g);
        return s;
    };
    cudaError_t ce = sweep_init_constants();
    if (ce != cudaSuccess) {
        set_error(std::string("constants: ") + cudaGetErrorString(ce));
        return fail(LPA_ECUDA);
    }
    const int64_t n = g->n, m = g->m;
    if ((st = dalloc(g, &g->off, (size_t)(n + 1))) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->idx, (size_t)m)) != LPA_OK) return fail(st);
    if (weights && (st = dalloc(g, &g->w, (size_t)m)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->C, (size_t)n)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->flags[0], (size_t)n)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->flags[1], (size_t)n)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->mover_v, (size_t)n)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->mover_v1, (size_t)n)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->mover_c, (size_t)n)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->mover_count, 2)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->fallbacks, 1)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->d_err, 8)) != LPA_OK) return fail(st);   // [0] error bits, [4..7] two counts
    if ((st = dalloc(g, &g->macc, 4)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->gdd, 1)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->rs_d, 1)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->queues, kQueueCount)) != LPA_OK) return fail(st);
    if ((st = dalloc(g, &g->active, 1)) != LPA_OK) return fail(st);
    if ((st = ensure_counters(g, 1, false)) != LPA_OK) return fail(st);

    cudaStream_t s = g->stream;
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        set_error(std::string(what) + ": " + cudaGetErrorString(e));
        return fail(e == cudaErrorMemoryAllocation ? LPA_ENOMEM : LPA_ECUDA);
    };
    cudaError_t e;
    if (flags & LPA_OFFSETS_I64) {
        e = cudaMemcpyAsync(g->off, offsets, (size_t)(n + 1) * sizeof(int64_t), kind, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy offsets");
    } else {
        int32_t *tmp = nullptr;
        if ((st = dalloc(g, &tmp, (size_t)(n + 1))) != LPA_OK) return fail(st);
        e = cudaMemcpyAsync(tmp, offsets, (size_t)(n + 1) * sizeof(int32_t), kind, s);
        if (e == cudaSuccess) {
            k_off32to64<<<grid_for(n + 1, 256, 16), 256, 0, s>>>(tmp, g->off, n + 1);
            e = cudaStreamSynchronize(s);
        }
        dfree(g, tmp);
        if (e != cudaSuccess) return cuda_fail(e, "copy offsets");
    }
    if (m > 0) {
        e = cudaMemcpyAsync(g->idx, indices, (size_t)m * sizeof(int32_t), kind, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy indices");
        if (weights) {
            e = cudaMemcpyAsync(g->w, weights, (size_t)m * sizeof(float), kind, s);
            if (e != cudaSuccess) return cuda_fail(e, "copy weights");
        }
    }
    // validation on the device (error bits and the two descent counts in one small block)
    cudaMemsetAsync(g->d_err, 0, 8 * sizeof(unsigned), s);
    k_validate<<<grid_for(std::max<int64_t>(n, m), 256, 16), 256, 0, s>>>(
        g->off, g->idx, g->w, n, m, g->d_err, reinterpret_cast<unsigned long long *>(g->d_err + 4));
    unsigned hv[8] = {0u, 0u, 0u, 0u, 0u, 0u, 1u, 0u};
    cudaMemcpyAsync(hv, g->d_err, sizeof(hv), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "validate");
    const unsigned err = hv[0];
    unsigned long long hdesc[2];
    memcpy(hdesc, hv + 4, sizeof(hdesc));
    g->rows_strict = hdesc[0] == hdesc[1];
    if (err) {
        std::string msg = "lpa_create: invalid graph:";
        if (err & 1) msg += " offsets decrease;";
        if (err & 2) msg += " offsets[0] != 0;";
        if (err & 4) msg += " offsets[n] != n_entries;";
        if (err & 8) msg += " index out of range;";
        if (err & 16) msg += " weight negative, NaN or Inf;";
        set_error(msg);
        return fail(LPA_EINVAL);
    }
    bool unit_weights = false;
    {
        // integer sums are exact when every weight is an integer and every row sum is below
        // 2^24: max weight x max degree below 2^24 settles it, else the exact row sums do
        unsigned long long *mk = nullptr;
        if ((st = dalloc(g, &mk, 2)) != LPA_OK) return fail(st);
        unsigned *fl = reinterpret_cast<unsigned *>(g->d_err);
        cudaMemsetAsync(mk, 0, 2 * sizeof(unsigned long long), s);
        const unsigned init[2] = {6u, 0u};            // flags, largest weight bits
        cudaMemcpyAsync(fl, init, sizeof(init), cudaMemcpyHostToDevice, s);
        if (g->w && m > 0)
            k_weight_flat<<<grid_for(m, 256, 16), 256, 0, s>>>(g->w, m, fl, fl + 1);
        k_degree_max<<<grid_for(n, 256, 16), 256, 0, s>>>(g->off, n, mk + 1);
        unsigned hf[2] = {0u, 0u};
        unsigned long long hd = 0;
        cudaMemcpyAsync(hf, fl, sizeof(hf), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&hd, mk + 1, sizeof(hd), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            dfree(g, mk);
            return cuda_fail(e, "weight properties");
        }
        float wmax = 1.0f;
        if (g->w) memcpy(&wmax, &hf[1], sizeof(float));
        const bool integral = (hf[0] & 2u) != 0;
        unit_weights = (hf[0] & 4u) != 0;
        if (integral && (double)wmax * (double)hd < 16777216.0) {
            g->int_weights = true;
        } else if (integral) {
            const unsigned two = 2u;
            cudaMemcpyAsync(fl, &two, sizeof(unsigned), cudaMemcpyHostToDevice, s);
            k_weight_props<<<grid_for(n * 32, 256, 16), 256, 0, s>>>(g->off, g->w, n, fl, mk);
            unsigned long long hk = 0;
            cudaMemcpyAsync(&hk, mk, sizeof(hk), cudaMemcpyDeviceToHost, s);
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                dfree(g, mk);
                return cuda_fail(e, "weight properties");
            }
            g->int_weights = hk < (1ull << 24);
        } else {
            g->int_weights = false;
        }
        dfree(g, mk);
    }
    if (flags & LPA_CHECK_SYMMETRIC) {
        unsigned long long *acc = nullptr;
        if ((st = dalloc(g, &acc, 4)) != LPA_OK) return fail(st);
        cudaMemsetAsync(acc, 0, 4 * sizeof(unsigned long long), s);
        k_symmetric<<<grid_for(n * 32, 256, 16), 256, 0, s>>>(g->off, g->idx, g->w, n, acc);
        unsigned long long h[4];
        cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        dfree(g, acc);
        if (e != cudaSuccess) return cuda_fail(e, "symmetry check");
        if (h[0] != h[1] || h[2] != h[3]) {
            set_error("lpa_create: graph is not undirected (entry (i,j,w) without (j,i,w))");
            return fail(LPA_EINVAL);
        }
    }
    if (unit_weights && g->w) {
        // every weight is exactly 1: the kernels take the unit-weight path (same sums, no
        // weight reads) and the device copy is released
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "weights");
        dfree(g, g->w);
        g->w = nullptr;
    }
    if ((st = build_buckets(g)) != LPA_OK) return fail(st);
    if ((st = init_state(g)) != LPA_OK) return fail(st);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "init");
    *out = g;
    return LPA_OK;
}

// Eq. 1 in two halves: the kernels that fill the graph's four accumulator words (no wait), and
// Q from those words once they are on the host (exact integers, or float64).
int graph_modularity_enqueue(lpa_graph *g)
{
    if (g->n == 0) return LPA_OK;
    if (!g->Sig) {
        LPA_CHECK(dalloc(g, &g->Sig, (size_t)g->n));
        LPA_CUDA(cudaMemsetAsync(g->Sig, 0, (size_t)g->n * sizeof(double), g->stream));
    }
    LPA_CUDA(cudaMemsetAsync(g->macc, 0, 4 * sizeof(double), g->stream));
    const int64_t *bs = g->bucket_start;
    const HubArgs &ha = g->gdh.hub;
    auto run_lists = [&](auto *Sig, auto *acc) {
        using ACC = std::remove_pointer_t<decltype(Sig)>;
        const int64_t n_small = bs[B_GROUP + 1] - bs[B_THREAD];
        const int64_t n_mid = bs[B_CTA_XL + 1] - bs[B_WARP];
        if (n_small > 0)
            k_mod_list<4, ACC><<<grid_for(n_small * 4, 256, 16), 256, 0, g->stream>>>(
                g->off, g->idx, g->w, g->C, g->lists + bs[B_THREAD], n_small, Sig, acc);
        if (n_mid > 0)
            k_mod_list<32, ACC><<<grid_for(n_mid * 32, 256, 16), 256, 0, g->stream>>>(
                g->off, g->idx, g->w, g->C, g->lists + bs[B_WARP], n_mid, Sig, acc);
        if (ha.n_hubs > 0 && ha.n_chunks > 0)
            k_mod_hub_chunks<ACC><<<(unsigned)ha.n_chunks, 256, 0, g->stream>>>(
                g->idx, g->w, g->C, ha.hub_v, ha.chunk_h, ha.chunk_e0, ha.chunk_e1, Sig, acc);
    };
    if (g->int_weights) {
        unsigned long long *SigU = reinterpret_cast<unsigned long long *>(g->Sig);
        unsigned long long *acc = reinterpret_cast<unsigned long long *>(g->macc);
        run_lists(SigU, acc);
        k_mod_sq_int<<<grid_for(g->n, 256, 16), 256, 0, g->stream>>>(SigU, g->n, acc);
    } else {
        run_lists(g->Sig, g->macc);
        k_mod_sq<<<grid_for(g->n, 256, 16), 256, 0, g->stream>>>(g->Sig, g->n, g->macc);
    }
    LPA_CUDA(cudaGetLastError());
    return LPA_OK;
}

double graph_modularity_finish(const lpa_graph *g, const void *acc_words)
{
    if (g->n == 0) return 0.0;
    if (g->int_weights) {
        const unsigned long long *h = static_cast<const unsigned long long *>(acc_words);
        const __int128 two_m = (__int128)h[1], in = (__int128)h[0];
        const __int128 sq = ((__int128)h[3] << 64) | (__int128)h[2];
        const __int128 num = two_m * in - sq, den = two_m * two_m;
        return (den == 0) ? 0.0 : (double)num / (double)den;
    }
    const double *h = static_cast<const double *>(acc_words);
    const double in = h[0], two_m = h[1], sq = h[2];
    return (two_m == 0.0) ? 0.0 : in / two_m - sq / (two_m * two_m);
}

int graph_modularity(lpa_graph *g, double *q)
{
    *q = 0.0;
    if (g->n == 0) return LPA_OK;
    LPA_CHECK(graph_modularity_enqueue(g));
    unsigned long long h[4];
    LPA_CUDA(cudaMemcpyAsync(h, g->macc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    LPA_CUDA(cudaStreamSynchronize(g->stream));
    *q = graph_modularity_finish(g, h);
    return LPA_OK;
}

}  // namespace lpa

// =======================================================================================
extern "C" {

const char *lpa_strerror(int status)
{
    switch (status) {
    case LPA_OK: return "success";
    case LPA_EINVAL: return "invalid argument";
    case LPA_ENOMEM: return "out of memory";
    case LPA_ECUDA: return "CUDA error";
    case LPA_ETIMEOUT: return "device wait timed out";
    case LPA_ESTATE: return "invalid state";
    case LPA_ECANCELED: return "request cancelled";
    default: return "unknown status";
    }
}

const char *lpa_last_error(void) { return t_error.c_str(); }

int lpa_trim_memory(void)
{
    std::lock_guard<std::mutex> lock(g_pool_mu);
    int prev = -1;
    cudaGetDevice(&prev);
    for (int d = 0; d < kMaxPoolDevices; ++d) {
        if (!g_pools[d]) continue;
        cudaSetDevice(d);
        cudaDeviceSynchronize();
        const cudaError_t e = cudaMemPoolTrimTo(g_pools[d], 0);
        if (e != cudaSuccess) {
            if (prev >= 0) cudaSetDevice(prev);
            set_error(std::string("lpa_trim_memory: ") + cudaGetErrorString(e));
            return LPA_ECUDA;
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    return LPA_OK;
}

void lpa_debug_fail_allocations(long long after) { g_alloc_budget.store(after < 0 ? -1 : after); }

const char *lpa_kernel_name(int slot)
{
    static const char *names[LPA_NUM_KERNELS] = {"thread", "group", "warp", "cta", "cta_large", "cta_xl",
                                                 "hub_begin", "hub_acc", "hub_clear", "hub_move", "hub_mark", "apply"};
    if (slot < 0 || slot >= LPA_NUM_KERNELS) return "";
    return names[slot];
}

int lpa_create(const void *offsets, const int32_t *indices, const float *weights, int64_t n_vertices,
               int64_t n_entries, int flags, void *cuda_stream, lpa_graph **out)
{
    return create_graph(offsets, indices, weights, n_vertices, n_entries, flags, (cudaStream_t)cuda_stream, nullptr,
                        nullptr, out);
}

void lpa_destroy(lpa_graph *g) { destroy_graph(g); }

int64_t lpa_num_vertices(const lpa_graph *g) { return g ? g->n : -1; }
int64_t lpa_num_entries(const lpa_graph *g) { return g ? g->m : -1; }
int64_t lpa_device_bytes(const lpa_graph *g) { return g ? g->bytes : -1; }

int lpa_set_stream(lpa_graph *g, void *cuda_stream)
{
    if (!g) return LPA_EINVAL;
    g->stream = (cudaStream_t)cuda_stream;
    return LPA_OK;
}

int lpa_get_tuning(const lpa_graph *g, lpa_tuning *t)
{
    if (!g || !t) return LPA_EINVAL;
    *t = g->tuning;
    return LPA_OK;
}

int lpa_set_tuning(lpa_graph *g, const lpa_tuning *t)
{
    if (!g || !t) return LPA_EINVAL;
    DeviceGuard dg(g->device);
    if (check_tuning(*t) != LPA_OK) {
        set_error("lpa_set_tuning: thresholds out of range, decreasing, or a table does not fit in shared memory");
        return LPA_EINVAL;
    }
    g->tuning = *t;
    return build_buckets(g);
}

int lpa_labels(const lpa_graph *g, int32_t *out, int64_t n, int out_on_device)
{
    if (!g || (!out && n > 0) || n != g->n) {
        set_error("lpa_labels: bad arguments");
        return LPA_EINVAL;
    }
    DeviceGuard dg(g->device);
    if (n == 0) return LPA_OK;
    LPA_CUDA(cudaMemcpyAsync(out, g->C, (size_t)n * sizeof(int32_t),
                             out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    LPA_CUDA(cudaStreamSynchronize(g->stream));
    return LPA_OK;
}

int lpa_get_state(const lpa_graph *g, int32_t *labels, uint8_t *unprocessed, int32_t *next_iter, int64_t n,
                  int on_device)
{
    if (!g || n != g->n) return LPA_EINVAL;
    DeviceGuard dg(g->device);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (labels && n) LPA_CUDA(cudaMemcpyAsync(labels, g->C, (size_t)n * 4, k, g->stream));
    if (unprocessed && n) LPA_CUDA(cudaMemcpyAsync(unprocessed, g->flags[g->active_buf], (size_t)n, k, g->stream));
    LPA_CUDA(cudaStreamSynchronize(g->stream));
    if (next_iter) *next_iter = g->next_iter;
    return LPA_OK;
}

int lpa_set_state(lpa_graph *g, const int32_t *labels, const uint8_t *unprocessed, int32_t next_iter, int64_t n,
                  int on_device)
{
    if (!g || n != g->n || next_iter < 0) {
        set_error("lpa_set_state: bad arguments");
        return LPA_EINVAL;
    }
    DeviceGuard dg(g->device);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (n == 0) {
        g->next_iter = next_iter;
        return LPA_OK;
    }
    // stage labels in the mover buffer and flags in the idle flag buffer, so that a rejected
    // state leaves the handle unchanged
    uint8_t *stage = g->flags[1 - g->active_buf];
    if (labels) LPA_CUDA(cudaMemcpyAsync(g->mover_v, labels, (size_t)n * 4, k, g->stream));
    else LPA_CUDA(cudaMemcpyAsync(g->mover_v, g->C, (size_t)n * 4, cudaMemcpyDeviceToDevice, g->stream));
    if (unprocessed) LPA_CUDA(cudaMemcpyAsync(stage, unprocessed, (size_t)n, k, g->stream));
    else LPA_CUDA(cudaMemcpyAsync(stage, g->flags[g->active_buf], (size_t)n, cudaMemcpyDeviceToDevice, g->stream));
    LPA_CUDA(cudaMemsetAsync(g->d_err, 0, 4, g->stream));
    k_check_state<<<grid_for(n, 256, 16), 256, 0, g->stream>>>(g->off, n, g->mover_v, stage, g->d_err);
    unsigned err = 0;
    LPA_CUDA(cudaMemcpyAsync(&err, g->d_err, 4, cudaMemcpyDeviceToHost, g->stream));
    LPA_CUDA(cudaStreamSynchronize(g->stream));
    if (err) {
        set_error("lpa_set_state: label outside [0, n)");
        return LPA_EINVAL;
    }
    LPA_CUDA(cudaMemcpyAsync(g->C, g->mover_v, (size_t)n * 4, cudaMemcpyDeviceToDevice, g->stream));
    g->active_buf = 1 - g->active_buf;
    LPA_CUDA(cudaStreamSynchronize(g->stream));
    g->next_iter = next_iter;
    return LPA_OK;
}

int lpa_set_labels(lpa_graph *g, const int32_t *labels, int64_t n, int on_device)
{
    if (!g || !labels || n != g->n) {
        set_error("lpa_set_labels: bad arguments");
        return LPA_EINVAL;
    }
    DeviceGuard dg(g->device);
    if (n == 0) {
        g->next_iter = 0;
        return LPA_OK;
    }
    // every vertex with an edge becomes unprocessed (flags staged in the idle buffer)
    uint8_t *stage = g->flags[1 - g->active_buf];
    k_init_labels<<<grid_for(g->n, 256, 16), 256, 0, g->stream>>>(g->off, g->n, g->mover_c, stage);
    LPA_CUDA(cudaGetLastError());
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LPA_CUDA(cudaMemcpyAsync(g->mover_v, labels, (size_t)n * 4, k, g->stream));
    LPA_CUDA(cudaMemsetAsync(g->d_err, 0, 4, g->stream));
    k_check_state<<<grid_for(n, 256, 16), 256, 0, g->stream>>>(g->off, n, g->mover_v, nullptr, g->d_err);
    unsigned err = 0;
    LPA_CUDA(cudaMemcpyAsync(&err, g->d_err, 4, cudaMemcpyDeviceToHost, g->stream));
    LPA_CUDA(cudaStreamSynchronize(g->stream));
    if (err) {
        set_error("lpa_set_labels: label outside [0, n)");
        return LPA_EINVAL;
    }
    LPA_CUDA(cudaMemcpyAsync(g->C, g->mover_v, (size_t)n * 4, cudaMemcpyDeviceToDevice, g->stream));
    g->active_buf = 1 - g->active_buf;
    LPA_CUDA(cudaStreamSynchronize(g->stream));
    g->next_iter = 0;
    return LPA_OK;
}

int lpa_modularity(const lpa_graph *gc, double *q)
{
    lpa_graph *g = const_cast<lpa_graph *>(gc);
    if (!g || !q) return LPA_EINVAL;
    DeviceGuard dg(g->device);
    return graph_modularity(g, q);
}

int lpa_run(lpa_graph *g, double tolerance, int max_iters, int pl_period, int mode, lpa_stats *stats)
{
    return lpa_run_cc(g, tolerance, max_iters, pl_period, 0, mode, stats);
}

int lpa_run_cc(lpa_graph *g, double tolerance, int max_iters, int pl_period, int cc_period, int mode,
               lpa_stats *stats)
{
    if (!g || max_iters < 0 || pl_period < 0 || cc_period < 0 || !std::isfinite(tolerance) ||
        ((mode & ~LPA_RESUME) != LPA_SYNC && (mode & ~LPA_RESUME) != LPA_ASYNC)) {
        set_error("lpa_run: bad arguments");
        return LPA_EINVAL;
    }
    if (cc_period > 0 && (mode & ~LPA_RESUME) != LPA_SYNC) {
        set_error("lpa_run_cc: the Cross-Check is available in the synchronous mode only");
        return LPA_EINVAL;
    }
    DeviceGuard dg(g->device);
    const bool async_mode = (mode & ~LPA_RESUME) == LPA_ASYNC;
    if (cc_period > 0 && !g->cc_word) {               // Cross-Check arrays, on first use
        LPA_CHECK(dalloc(g, &g->cc_prev, (size_t)std::max<int64_t>(g->n, 1)));
        LPA_CHECK(dalloc(g, &g->cc_midx, (size_t)std::max<int64_t>(g->n, 1)));
        LPA_CHECK(dalloc(g, &g->cc_par0, (size_t)std::max<int64_t>(g->n, 1)));
        LPA_CHECK(dalloc(g, &g->cc_word, (size_t)std::max<int64_t>(g->n, 1)));
        LPA_CHECK(dalloc(g, &g->cc_ctr, (size_t)(kCcPasses + 1)));
        LPA_CUDA(cudaMemsetAsync(g->cc_midx, 0xFF, (size_t)std::max<int64_t>(g->n, 1) * sizeof(int32_t), g->stream));
        LPA_CHECK(upload_descriptor(g));
    }
    cudaStream_t s = g->stream;
    const bool timing = stats && stats->time_kernels;
    if (stats) {
        const int32_t tk = stats->time_kernels;
        memset(stats, 0, sizeof(*stats));
        stats->time_kernels = tk;
    }
    if (!(mode & LPA_RESUME)) LPA_CHECK(init_state(g));
    const int start = g->next_iter;
    if (stats) {
        stats->first_iter = start;
        stats->iterations = start;
    }
    if (g->n == 0 || start >= max_iters) {
        LPA_CUDA(cudaStreamSynchronize(s));
        return LPA_OK;
    }
    const int span = max_iters - start;
    LPA_CHECK(ensure_counters(g, span, true));
    if (!g->hm) {
        if (cudaMallocHost((void **)&g->hm, sizeof(lpa_graph::HostMirror)) != cudaSuccess) {
            cudaGetLastError();
            g->hm = nullptr;
            set_error("cudaMallocHost failed");
            return LPA_ENOMEM;
        }
    }
    LPA_CHECK(upload_descriptor(g));
    LPA_CUDA(cudaMemsetAsync(g->ctr, 0, (size_t)kPerSweep * span * sizeof(unsigned long long), s));
    LPA_CUDA(cudaMemsetAsync(g->fallbacks, 0, sizeof(unsigned long long), s));
    LPA_CUDA(cudaMemsetAsync(g->mover_count, 0, 2 * sizeof(unsigned long long), s));
    // the unprocessed flags of sweep `start` must sit where the kernels read them
    const int target = async_mode ? 0 : (start & 1);
    if (g->active_buf != target)
        LPA_CUDA(cudaMemcpyAsync(g->flags[target], g->flags[g->active_buf], (size_t)g->n, cudaMemcpyDeviceToDevice, s));
    if (!async_mode) LPA_CUDA(cudaMemsetAsync(g->flags[1 - target], 0, (size_t)g->n, s));
    g->active_buf = target;
    RunState &rs = g->hm->rs;
    rs = RunState{};
    rs.l = start;
    rs.first = start;
    rs.max_iters = max_iters;
    rs.pl_period = pl_period;
    rs.async_mode = async_mode ? 1 : 0;
    // a fresh synchronous run starts without marks (the first sweep moves most vertices); a
    // resumed run starts from its processed flags; Cross-Check runs always mark
    rs.mark = (async_mode || (mode & LPA_RESUME) || cc_period > 0) ? 1 : 0;
    rs.cc_period = cc_period;
    rs.tol = tolerance;
    rs.n = g->n;
    rs.fresh = (mode & LPA_RESUME) ? 0 : 1;
    rs.adaptive = 1;
    g->hm->active = 1;
    LPA_CUDA(cudaMemcpyAsync(g->rs_d, &g->hm->rs, sizeof(RunState), cudaMemcpyHostToDevice, s));
    LPA_CUDA(cudaMemcpyAsync(g->active, &g->hm->active, sizeof(int32_t), cudaMemcpyHostToDevice, s));

    SweepPlan p{};
    p.gd = g->gdd;
    p.n_graphs = 1;
    for (int b = B_THREAD; b <= B_CTA_XL; ++b) {
        p.items[b] = g->items_at[b];
        p.n_items[b] = (int32_t)g->items_h[b].size();
        p.n_vertices[b] = g->bucket_start[b + 1] - g->bucket_start[b];
    }
    plan_slots(g->tuning, p.slots);
    for (int q = 0; q < HL_COUNT; ++q) {
        p.hub_items[q] = g->hub_items_d[q];
        p.n_hub_items[q] = (int32_t)g->hub_items_h[q].size();
    }
    p.per_graph = g->per_graph_d;
    p.queues = g->queues;
    p.active_count = g->active;
    p.group_lanes = g->tuning.group_lanes;
    p.flat_buckets = g->tuning.flat_buckets;
    p.cta_threads = g->tuning.cta_threads;
    p.cta_large_threads = g->tuning.cta_large_threads;
    p.cta_xl_threads = g->tuning.cta_xl_threads;
    p.hub_chunk = g->tuning.hub_chunk;
    p.int_weights = plan_int_weights(g) ? 1 : 0;
    p.probe = g->tuning.probe;
    p.cc_any = cc_period > 0 ? 1 : 0;
    p.cc_ctr = g->cc_ctr;
    p.f64 = g->tuning.float_values == 2 ? 1 : 0;

    size_t evn = 0;
    cudaEvent_t run0 = event_at(g, evn++), run1 = event_at(g, evn++);
    if (!run0 || !run1) {
        set_error("cudaEventCreate failed");
        return LPA_ECUDA;
    }
    EventHook hook(g, &evn);
    std::vector<std::pair<size_t, size_t>> iter_ev;
    int launches = 0;
    LPA_CUDA(cudaEventRecord(run0, s));
    int ran = 0;
    for (; ran < span; ++ran) {
        const size_t ie0 = evn++, ie1 = evn++;
        if (!event_at(g, ie1)) return LPA_ECUDA;
        hook.iter = ran;
        hook.on = timing && ran < LPA_STATS_MAX_ITERS;
        LPA_CUDA(cudaEventRecord(g->events[ie0], s));
        p.pull_mode = g->hm->rs.pull ? 1 : 0;           // the state read back after the last sweep
        LPA_CUDA(enqueue_sweep(p, s, &hook, &launches));
        LPA_CUDA(cudaEventRecord(g->events[ie1], s));
        iter_ev.push_back({ie0, ie1});
        LPA_CUDA(cudaMemcpyAsync(&g->hm->rs, g->rs_d, sizeof(RunState), cudaMemcpyDeviceToHost, s));
        LPA_CUDA(cudaStreamSynchronize(s));
        if (g->hm->rs.cc_unresolved) {
            set_error("lpa_run_cc: the Cross-Check resolution did not finish");
            return LPA_ESTATE;
        }
        if (g->hm->rs.done) {
            ++ran;
            break;
        }
    }
    LPA_CUDA(cudaEventRecord(run1, s));
    unsigned long long fb = 0;
    LPA_CUDA(cudaMemcpyAsync(&fb, g->fallbacks, sizeof(fb), cudaMemcpyDeviceToHost, s));
    LPA_CUDA(cudaMemcpyAsync(g->h_ctr, g->ctr, (size_t)kPerSweep * ran * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, s));
    LPA_CUDA(cudaStreamSynchronize(s));
    const int l_end = g->hm->rs.l;
    g->next_iter = l_end;
    g->active_buf = async_mode ? 0 : (l_end & 1);
    if (stats) {
        stats->iterations = l_end;
        stats->converged = g->hm->rs.converged;
        stats->probe_fallbacks = (int64_t)fb;
        stats->launches = launches;
        cudaEventElapsedTime(&stats->total_ms, run0, run1);
        for (int r = 0; r < ran && r < LPA_STATS_MAX_ITERS; ++r) {
            const unsigned long long *hc = g->h_ctr + (size_t)kPerSweep * r;
            int64_t act = 0, edg = 0, mv = 0, mk = 0;
            for (int k = 0; k < LPA_NUM_KERNELS; ++k) {
                act += (int64_t)hc[k * kCtrFields + CTR_ACTIVE];
                edg += (int64_t)hc[k * kCtrFields + CTR_EDGES];
                mv += (int64_t)hc[k * kCtrFields + CTR_MOVED];
                mk += (int64_t)hc[k * kCtrFields + CTR_MARKS];
                stats->kernel_edges[r][k] = (int64_t)hc[k * kCtrFields + CTR_EDGES];
                stats->kernel_active[r][k] = (int64_t)hc[k * kCtrFields + CTR_ACTIVE];
            }
            stats->changed[r] = mv;
            stats->active[r] = act;
            stats->edges[r] = edg;
            stats->marks[r] = mk;
            cudaEventElapsedTime(&stats->iter_ms[r], g->events[iter_ev[r].first], g->events[iter_ev[r].second]);
        }
        for (const auto &r : hook.recs) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, g->events[r.e0], g->events[r.e1]);
            stats->kernel_ms[r.iter][r.slot] += ms;
        }
    }
    return LPA_OK;
}

size_t lpa_struct_size(int which)
{
    switch (which) {
    case 0: return sizeof(lpa_stats);
    case 1: return sizeof(lpa_tuning);
    default: return 0;
    }
}

}  // extern "C"
