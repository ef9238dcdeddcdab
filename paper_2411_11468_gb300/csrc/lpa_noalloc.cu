// lpa_modularity_noalloc: modularity (Eq. 1) of a caller-owned, labelled CSR graph that makes
// no device allocation.  Some callers cannot call cudaMalloc: code that runs while another
// framework owns the device memory pool (and forbids outside allocations), callers inside a
// memory-constrained service that has already reserved all device memory, or code paths that
// must not hit the allocator's synchronisation.  This entry point uses a fixed scratch array
// compiled into the library instead of any allocation.
//
// The scratch is a file-scope __device__ array: every GPU that loads the library holds it
// until the process exits, and every call on that GPU shares it.  Calls that overlap on the
// GPU (different streams, or different host threads) race on it and give wrong results; the
// caller must order them.  Each call clears the part it uses before use.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lpa_internal.h"

namespace {

constexpr int64_t kMaxVertices = LPA_NOALLOC_MAX_VERTICES;
constexpr int kAccWords = 8;      // accumulators after the Sigma part: sigma_in, 2m, sum Sigma^2, error

// Sigma_c for labels c < kMaxVertices, followed by kAccWords accumulators.  In host code this
// name is only a stand-in for the symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kMaxVertices + kAccWords];

// Device address of the scratch array on the current device.  Looked up on every call (a
// cheap query next to the call's two stream synchronisations), so no address outlives the
// context it was taken in.
cudaError_t scratch_address(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

// Checks the CSR and the labels before anything is indexed by them; bits as lpa_create's
// validation (1 offsets decrease, 2 offsets[0] != 0, 4 offsets[n] != m, 8 index out of range,
// 16 bad weight) plus 32 for a label outside [0, n).
__global__ void k_na_validate(const int64_t *off, const int32_t *idx, const float *w, const int32_t *C, int64_t n,
                              int64_t m, unsigned long long *err)
{
    unsigned long long bad = 0;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (tid == 0) {
        if (off[0] != 0) bad |= 2;
        if (off[n] != m) bad |= 4;
    }
    for (int64_t i = tid; i < n; i += stride) {
        if (off[i] > off[i + 1]) bad |= 1;
        if (C[i] < 0 || (int64_t)C[i] >= n) bad |= 32;
    }
    for (int64_t e = tid; e < m; e += stride) {
        if (idx[e] < 0 || (int64_t)idx[e] >= n) bad |= 8;
        if (w && !(isfinite(w[e]) && w[e] >= 0.0f)) bad |= 16;
    }
    if (bad) atomicOr(err, bad);
}

// A warp per row: K_i and the weight of entries whose neighbour shares the label, in float64;
// Sigma_{C_i} += K_i.  Runs only after validation passed.
__global__ void __launch_bounds__(256) k_na_rows(const int64_t *off, const int32_t *idx, const float *w,
                                                 const int32_t *C, int64_t n, double *sig, double *acc)
{
    __shared__ double s_in[8], s_k[8];
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double tin = 0.0, tk = 0.0;
    for (int64_t i = warp; i < n; i += nwarps) {
        const int64_t o0 = off[i], o1 = off[i + 1];
        if (o0 == o1) continue;
        const int32_t ci = C[i];
        double k = 0.0, in = 0.0;
        for (int64_t e = o0 + lane; e < o1; e += 32) {
            const double we = w ? (double)w[e] : 1.0;
            k += we;
            if (C[idx[e]] == ci) in += we;
        }
        k = warp_sum(k);
        in = warp_sum(in);
        if (lane == 0) {
            atomicAdd(sig + ci, k);
            tin += in;
            tk += k;
        }
    }
    if (lane == 0) {
        s_in[threadIdx.x >> 5] = tin;
        s_k[threadIdx.x >> 5] = tk;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int q = 0; q < 8; ++q) {
            a += s_in[q];
            b += s_k[q];
        }
        atomicAdd(acc + 0, a);
        atomicAdd(acc + 1, b);
    }
}

__global__ void __launch_bounds__(256) k_na_squares(const double *sig, int64_t n, double *acc)
{
    __shared__ double s[8];
    double t = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        t += sig[c] * sig[c];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int q = 0; q < 8; ++q) a += s[q];
        atomicAdd(acc + 2, a);
    }
}

int blocks_for(int64_t work)
{
    int64_t b = (work + 255) / 256;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

extern "C" int lpa_modularity_noalloc(const int64_t *offsets, const int32_t *indices, const float *weights,
                                      const int32_t *labels, int64_t n_vertices, int64_t n_entries,
                                      void *cuda_stream, double *q)
{
    if (!q || !offsets || n_vertices < 0 || n_entries < 0 || (n_vertices > 0 && !labels) ||
        (n_entries > 0 && !indices)) {
        lpa::set_error("lpa_modularity_noalloc: bad arguments");
        return LPA_EINVAL;
    }
    if (n_vertices > kMaxVertices) {
        lpa::set_error("lpa_modularity_noalloc: n_vertices " + std::to_string(n_vertices) +
                       " exceeds the fixed scratch limit of " + std::to_string(kMaxVertices) +
                       " vertices; use lpa_modularity on a graph handle instead");
        return LPA_EINVAL;
    }
    *q = 0.0;
    if (n_vertices == 0) return LPA_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) {
        lpa::set_error(std::string("lpa_modularity_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return LPA_ECUDA;
    }
    double *sig = scratch;
    double *acc = scratch + kMaxVertices;
    unsigned long long *err = reinterpret_cast<unsigned long long *>(acc + 3);
    // the previous call's contents stay in the array: clear the part this call reads
    e = cudaMemsetAsync(sig, 0, (size_t)n_vertices * sizeof(double), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, kAccWords * sizeof(double), s);
    if (e == cudaSuccess) {
        k_na_validate<<<blocks_for(n_vertices > n_entries ? n_vertices : n_entries), 256, 0, s>>>(
            offsets, indices, weights, labels, n_vertices, n_entries, err);
        e = cudaGetLastError();
    }
    unsigned long long herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        lpa::set_error(std::string("lpa_modularity_noalloc: ") + cudaGetErrorString(e));
        return LPA_ECUDA;
    }
    if (herr) {
        lpa::set_error("lpa_modularity_noalloc: invalid graph or labels (validation bits " + std::to_string(herr) + ")");
        return LPA_EINVAL;
    }
    k_na_rows<<<blocks_for(n_vertices * 32), 256, 0, s>>>(offsets, indices, weights, labels, n_vertices, sig, acc);
    k_na_squares<<<blocks_for(n_vertices), 256, 0, s>>>(sig, n_vertices, acc);
    double h[3];
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        lpa::set_error(std::string("lpa_modularity_noalloc: ") + cudaGetErrorString(e));
        return LPA_ECUDA;
    }
    const double in = h[0], two_m = h[1], sq = h[2];
    *q = (two_m == 0.0) ? 0.0 : in / two_m - sq / (two_m * two_m);
    return LPA_OK;
}
