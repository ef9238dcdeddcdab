/* Multicore CPU baseline for nu-LPA -- TEST AND BENCHMARK INFRASTRUCTURE, not the product.
 *
 * The synchronous sweep of Algorithm 1 (lpa / lpaMove, Eq. 3, Section 4 items 2-5) run
 * over OpenMP threads, in the style of the paper's multicore predecessor GVE-LPA (Section 2):
 * vertices are shared out dynamically; each thread gathers a vertex's neighbour label weights
 * in its own open-addressing table (linear probing, cleared through the list of used slots)
 * and takes the largest weight with the smallest label on ties.  It computes the same result
 * as the single-threaded oracle (`lpa_oracle.c`), which the tests check, and is timed by the
 * benchmark as a stronger CPU comparison than the oracle.  Shares no code with the oracle or
 * with the CUDA path.  Built with gcc -fopenmp.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t *key;      /* [cap], -1 = empty */
    float *sum;        /* [cap] */
    int32_t *used;     /* slots taken for the current vertex */
    uint32_t mask;     /* cap - 1 */
} mc_table;

static int mc_table_alloc(mc_table *t, int64_t dmax)
{
    uint64_t cap = 16;
    while (cap < 2 * (uint64_t)(dmax > 0 ? dmax : 1)) cap <<= 1;
    t->key = (int32_t *)malloc(cap * sizeof(int32_t));
    t->sum = (float *)malloc(cap * sizeof(float));
    t->used = (int32_t *)malloc(cap * sizeof(int32_t));
    t->mask = (uint32_t)(cap - 1);
    if (!t->key || !t->sum || !t->used) return -1;
    for (uint64_t s = 0; s < cap; ++s) t->key[s] = -1;
    return 0;
}

static void mc_table_free(mc_table *t)
{
    free(t->key);
    free(t->sum);
    free(t->used);
}

/* Largest-weight neighbour label of vertex i (smallest label among equal weights), or -1
 * when i has no neighbour other than itself. */
static int32_t mc_best(int64_t i, const int64_t *off, const int32_t *idx, const float *w, const int32_t *C,
                       mc_table *t)
{
    int64_t nu = 0;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        const int32_t j = idx[e];
        if (j == i) continue;
        const int32_t c = C[j];
        uint32_t s = ((uint32_t)c * 2654435761u) & t->mask;
        while (t->key[s] != c && t->key[s] != -1) s = (s + 1) & t->mask;
        if (t->key[s] == -1) {
            t->key[s] = c;
            t->sum[s] = 0.0f;
            t->used[nu++] = (int32_t)s;
        }
        t->sum[s] += w ? w[e] : 1.0f;
    }
    int32_t best = -1;
    float bw = 0.0f;
    for (int64_t u = 0; u < nu; ++u) {
        const int32_t s = t->used[u];
        const int32_t c = t->key[s];
        const float x = t->sum[s];
        if (best < 0 || x > bw || (x == bw && c < best)) {
            best = c;
            bw = x;
        }
        t->key[s] = -1;
    }
    return best;
}

int mc_threads(void) { return omp_get_max_threads(); }

/* Same arguments and meaning as orc_lpa_sync (synchronous, double-buffered labels and
 * processed flags; dN and edges indexed by absolute iteration), plus the thread count
 * (<= 0: all). */
int mc_lpa_sync(int64_t n, const int64_t *off, const int32_t *idx, const float *w, double tol, int max_iters,
                int pl_period, int start_iter, int32_t *C, uint8_t *active, int64_t *dN, int32_t *iters,
                int32_t *converged, int64_t *edges, int threads)
{
    *converged = 0;
    *iters = start_iter;
    if (n <= 0) return 0;
    if (threads > 0) omp_set_num_threads(threads);
    int64_t dmax = 0;
    for (int64_t i = 0; i < n; ++i)
        if (off[i + 1] - off[i] > dmax) dmax = off[i + 1] - off[i];
    int32_t *Cn = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *an = (uint8_t *)malloc((size_t)n);
    const int nt = omp_get_max_threads();
    mc_table *tabs = (mc_table *)calloc((size_t)nt, sizeof(mc_table));
    int bad = !Cn || !an || !tabs;
    for (int t = 0; t < nt && !bad; ++t) bad = mc_table_alloc(&tabs[t], dmax) != 0;
    if (bad) {
        if (tabs)
            for (int t = 0; t < nt; ++t) mc_table_free(&tabs[t]);
        free(tabs);
        free(Cn);
        free(an);
        return -1;
    }
    for (int l = start_iter; l < max_iters; ++l) {
        const int pl = (pl_period > 0) && (l % pl_period == 0);
        memcpy(Cn, C, (size_t)n * sizeof(int32_t));
        memset(an, 0, (size_t)n);
        int64_t changed = 0, scanned = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : changed, scanned)
        for (int64_t i = 0; i < n; ++i) {
            if (!active[i]) continue;
            scanned += off[i + 1] - off[i];
            mc_table *t = &tabs[omp_get_thread_num()];
            const int32_t c = mc_best(i, off, idx, w, C, t);
            if (c < 0) continue;
            const int32_t cur = C[i];
            if (c != cur && (!pl || c < cur)) {
                Cn[i] = c;
                ++changed;
                for (int64_t e = off[i]; e < off[i + 1]; ++e) __atomic_store_n(&an[idx[e]], (uint8_t)1, __ATOMIC_RELAXED);
            }
        }
        memcpy(C, Cn, (size_t)n * sizeof(int32_t));
        memcpy(active, an, (size_t)n);
        dN[l] = changed;
        if (edges) edges[l] = scanned;
        *iters = l + 1;
        if (!pl && (double)changed / (double)n < tol) {
            *converged = 1;
            break;
        }
    }
    for (int t = 0; t < nt; ++t) mc_table_free(&tabs[t]);
    free(tabs);
    free(Cn);
    free(an);
    return 0;
}
