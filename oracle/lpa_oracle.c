/*
 * CPU oracle for nu-LPA label propagation (Sahu, "nu-LPA: Fast GPU-based Label
 * Propagation Algorithm (LPA) for Community Detection", arXiv 2411.11468).
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It shares no
 * code with the CUDA path.  Plain single-threaded C11, written for readability:
 * every function states the passage of the paper it follows.
 *
 * Conventions (readings of the paper fixed for this project):
 *  - Labels are int32 vertex ids; the empty hashtable key is -1.
 *  - Eq. 3 (LPA update rule) with the smallest label among the max-weight labels
 *    (the paper's "strict LPA" picks "the first" max label; "first" is read as
 *    "smallest").  Candidates are the labels of the non-self neighbours.
 *  - Label weights are accumulated in float32, the paper's hashtable value type
 *    (Section 4.4 and the Configuration paragraph); with integer weights and
 *    K_i < 2^24 every partial sum is exact.
 *  - Pick-Less (Section 4.1, Algorithm 1): on iterations l with l mod rho == 0
 *    (l 0-based, rho = pl_period, 0 disables) a vertex may only move to a strictly
 *    smaller label.
 *  - Pruning (Section 4, item 4; Algorithm 1): a processed vertex is marked
 *    processed; a vertex that changes label marks every neighbour unprocessed.
 *  - Stop rule (Algorithm 1): after iteration l, stop when PL is off and
 *    dN / N < tolerance (strict, in double); at most max_iters iterations.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EMPTY (-1)

/* ---------------------------------------------------------------------------
 * Label weights by sort-and-count (Preliminaries: K_{i->c} = sum_{j in J_i, C_j = c} w_ij).
 * Self-loops are skipped as in Algorithm 1 ("if j = i continue").
 */
typedef struct {
    int32_t label;
    int64_t pos;
    float w;
} orc_item;

static int orc_item_cmp(const void *a, const void *b)
{
    const orc_item *x = (const orc_item *)a, *y = (const orc_item *)b;
    if (x->label != y->label) return x->label < y->label ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

/* Writes the distinct neighbour labels of vertex i (ascending) and their float32
 * weight sums; returns how many.  `scratch` holds at least D_i items. */
int64_t orc_label_weights(int64_t i, const int64_t *off, const int32_t *idx, const float *w,
                          const int32_t *C, int32_t *out_labels, float *out_sums, orc_item *scratch)
{
    int64_t cnt = 0;
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
        int32_t j = idx[e];
        if (j == i) continue;
        scratch[cnt].label = C[j];
        scratch[cnt].pos = e;
        scratch[cnt].w = w ? w[e] : 1.0f;
        ++cnt;
    }
    qsort(scratch, (size_t)cnt, sizeof(orc_item), orc_item_cmp);
    int64_t nd = 0;
    for (int64_t k = 0; k < cnt; ++k) {
        if (nd == 0 || out_labels[nd - 1] != scratch[k].label) {
            out_labels[nd] = scratch[k].label;
            out_sums[nd] = 0.0f;
            ++nd;
        }
        out_sums[nd - 1] += scratch[k].w;
    }
    return nd;
}

/* Eq. 3 with the smallest-label tie-break: argmax_c K_{i->c}; -1 when vertex i has
 * no non-self neighbour (no candidate label). */
int32_t orc_best_label(int64_t i, const int64_t *off, const int32_t *idx, const float *w,
                       const int32_t *C, int32_t *lab, float *sum, orc_item *scratch)
{
    int64_t nd = orc_label_weights(i, off, idx, w, C, lab, sum, scratch);
    int32_t best = -1;
    float bw = 0.0f;
    for (int64_t k = 0; k < nd; ++k) {          /* labels ascending: keep the first max */
        if (best < 0 || sum[k] > bw) {
            best = lab[k];
            bw = sum[k];
        }
    }
    return best;
}

static int64_t orc_max_degree(int64_t n, const int64_t *off)
{
    int64_t d = 0;
    for (int64_t i = 0; i < n; ++i)
        if (off[i + 1] - off[i] > d) d = off[i + 1] - off[i];
    return d;
}

typedef struct {
    int32_t *lab;
    float *sum;
    orc_item *scratch;
} orc_work;

static int orc_work_alloc(orc_work *wk, int64_t dmax)
{
    size_t k = (size_t)(dmax > 0 ? dmax : 1);
    wk->lab = (int32_t *)malloc(k * sizeof(int32_t));
    wk->sum = (float *)malloc(k * sizeof(float));
    wk->scratch = (orc_item *)malloc(k * sizeof(orc_item));
    return (wk->lab && wk->sum && wk->scratch) ? 0 : -1;
}

static void orc_work_free(orc_work *wk)
{
    free(wk->lab);
    free(wk->sum);
    free(wk->scratch);
}

/* ---------------------------------------------------------------------------
 * Synchronous LPA: every vertex of iteration l reads the labels and the active set
 * that iteration l-1 left (double buffered).  The paper's method is asynchronous;
 * this deterministic variant applies the same per-vertex step (Algorithm 1, lpaMove)
 * and the same driver loop (Algorithm 1, lpa) to frozen inputs.
 *
 * C [n]       in: labels at iteration start_iter; out: final labels.
 * active [n]  in: active set at start_iter (1 = unprocessed); out: the set for the
 *             next iteration.
 * dN [max_iters] out: changed-vertex counts, indexed by absolute iteration.
 * edges [max_iters] out (nullable): CSR entries of the vertices each iteration processed.
 * *iters out: index of the next iteration (= last iteration run + 1).
 * *converged out: 1 when the tolerance test stopped the loop.
 * Returns 0, or -1 on allocation failure.
 */
/* Cross-Check (Section 4.1), after the sweep that moved some vertices from Cprev to C:
 * a move of i to c* = C[i] is good when vertex c* is in community c* (C[c*] = c*); a bad
 * move reverts i to Cprev[i].  The paper reverts atomically, so that the two vertices of a
 * swap do not both revert; this reading checks the moved vertices in increasing id order
 * against the labels as they stand, earlier reverts included.  Returns the number of
 * reverted moves.  Marks made during the sweep stay. */
int64_t orc_cross_check(int64_t n, int32_t *C, const int32_t *Cprev)
{
    int64_t reverted = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (C[i] == Cprev[i]) continue;
        const int32_t c = C[i];
        if (C[c] != c) {
            C[i] = Cprev[i];
            ++reverted;
        }
    }
    return reverted;
}

/* Synchronous LPA with Pick-Less every pl_period sweeps (Section 4.1; 0: never) and
 * Cross-Check after every cc_period-th sweep (0: never): both on sweeps l with
 * l mod period = 0, so pl_period = cc_period > 0 is the paper's Hybrid.  dN counts the moves
 * that remain after the Cross-Check. */
int orc_lpa_sync_cc(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                    double tol, int max_iters, int pl_period, int cc_period, int start_iter,
                    int32_t *C, uint8_t *active, int64_t *dN, int32_t *iters, int32_t *converged,
                    int64_t *edges)
{
    *converged = 0;
    *iters = start_iter;
    if (n <= 0) return 0;
    orc_work wk;
    int32_t *Cn = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *an = (uint8_t *)malloc((size_t)n);
    if (!Cn || !an || orc_work_alloc(&wk, orc_max_degree(n, off)) != 0) {
        free(Cn);
        free(an);
        return -1;
    }
    for (int l = start_iter; l < max_iters; ++l) {
        int pl = (pl_period > 0) && (l % pl_period == 0);
        memcpy(Cn, C, (size_t)n * sizeof(int32_t));
        memset(an, 0, (size_t)n);
        int64_t changed = 0, scanned = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (!active[i]) continue;
            scanned += off[i + 1] - off[i];
            int32_t c = orc_best_label(i, off, idx, w, C, wk.lab, wk.sum, wk.scratch);
            if (c < 0) continue;
            int32_t cur = C[i];
            if (c != cur && (!pl || c < cur)) {
                Cn[i] = c;
                ++changed;
                for (int64_t e = off[i]; e < off[i + 1]; ++e) an[idx[e]] = 1;
            }
        }
        if (cc_period > 0 && l % cc_period == 0) changed -= orc_cross_check(n, Cn, C);
        memcpy(C, Cn, (size_t)n * sizeof(int32_t));
        memcpy(active, an, (size_t)n);   /* processed vertices are cleared, marks set */
        dN[l] = changed;
        if (edges) edges[l] = scanned;
        *iters = l + 1;
        if (!pl && (double)changed / (double)n < tol) {
            *converged = 1;
            break;
        }
    }
    free(Cn);
    free(an);
    orc_work_free(&wk);
    return 0;
}

int orc_lpa_sync(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                 double tol, int max_iters, int pl_period, int start_iter,
                 int32_t *C, uint8_t *active, int64_t *dN, int32_t *iters, int32_t *converged,
                 int64_t *edges)
{
    return orc_lpa_sync_cc(n, off, idx, w, tol, max_iters, pl_period, 0, start_iter, C, active, dN, iters,
                           converged, edges);
}

/* Asynchronous LPA in the paper's sense (Section 4, item 1): one label vector and one
 * flag vector, both updated in place.  Vertices are visited in the fixed order
 * 0..n-1, so the result is one particular schedule of the paper's racy sweep. */
int orc_lpa_async(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                  double tol, int max_iters, int pl_period, int start_iter,
                  int32_t *C, uint8_t *active, int64_t *dN, int32_t *iters, int32_t *converged,
                  int64_t *edges)
{
    *converged = 0;
    *iters = start_iter;
    if (n <= 0) return 0;
    orc_work wk;
    if (orc_work_alloc(&wk, orc_max_degree(n, off)) != 0) return -1;
    for (int l = start_iter; l < max_iters; ++l) {
        int pl = (pl_period > 0) && (l % pl_period == 0);
        int64_t changed = 0, scanned = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (!active[i]) continue;
            active[i] = 0;                                  /* mark processed */
            scanned += off[i + 1] - off[i];
            int32_t c = orc_best_label(i, off, idx, w, C, wk.lab, wk.sum, wk.scratch);
            if (c < 0) continue;
            int32_t cur = C[i];
            if (c != cur && (!pl || c < cur)) {
                C[i] = c;
                ++changed;
                for (int64_t e = off[i]; e < off[i + 1]; ++e) active[idx[e]] = 1;
            }
        }
        dN[l] = changed;
        if (edges) edges[l] = scanned;
        *iters = l + 1;
        if (!pl && (double)changed / (double)n < tol) {
            *converged = 1;
            break;
        }
    }
    orc_work_free(&wk);
    return 0;
}

/* Asynchronous LPA under a wave schedule: a reading of Section 4 item 1 for a sweep that
 * many threads run at once.  Each sweep visits the waves 0, 1, ..., n_waves - 1 in turn.
 * Vertex i takes its processed flag (reads it and marks itself processed) when wave
 * take_of[i] starts, and decides in wave wave_of[i] >= take_of[i]: if its flag was set when
 * taken, it computes c* from the labels as they stand when its deciding wave starts (no
 * vertex of a wave sees another's move of the same wave).  The moves of a wave and the
 * neighbour marks of its movers take effect when the wave ends.  take_of = NULL takes every
 * flag in the vertex's deciding wave.  So a schedule of one vertex per wave in id order is
 * orc_lpa_async, and one wave holding every vertex is orc_lpa_sync; a parallel sweep sits
 * between the two.  Pick-Less and the stop rule are those of Algorithm 1.  Returns 0, -1 on
 * allocation failure, -2 for a wave index outside [0, n_waves) or a take after the decision. */
static int orc_bucket_by(int64_t n, const int32_t *key, int32_t n_keys, int64_t **first_out, int64_t **member_out)
{
    int64_t *first = (int64_t *)calloc((size_t)n_keys + 1, sizeof(int64_t));
    int64_t *member = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc((size_t)n_keys * sizeof(int64_t));
    if (!first || !member || !fill) {
        free(first);
        free(member);
        free(fill);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) ++first[key[i] + 1];
    for (int32_t q = 0; q < n_keys; ++q) first[q + 1] += first[q];
    memcpy(fill, first, (size_t)n_keys * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) member[fill[key[i]]++] = i;     /* ascending ids per key */
    free(fill);
    *first_out = first;
    *member_out = member;
    return 0;
}

int orc_lpa_async_waves(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                        double tol, int max_iters, int pl_period, int start_iter,
                        const int32_t *wave_of, const int32_t *take_of, int32_t n_waves,
                        int32_t *C, uint8_t *active, int64_t *dN, int32_t *iters, int32_t *converged,
                        int64_t *edges)
{
    *converged = 0;
    *iters = start_iter;
    if (n <= 0) return 0;
    const int32_t *take = take_of ? take_of : wave_of;
    for (int64_t i = 0; i < n; ++i)
        if (wave_of[i] < 0 || wave_of[i] >= n_waves || take[i] < 0 || take[i] > wave_of[i]) return -2;
    int64_t *first = NULL, *member = NULL, *tfirst = NULL, *tmember = NULL;
    int32_t *newc = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint8_t *taken = (uint8_t *)malloc((size_t)n);
    orc_work wk;
    int bad = !newc || !taken || orc_bucket_by(n, wave_of, n_waves, &first, &member) != 0 ||
              orc_bucket_by(n, take, n_waves, &tfirst, &tmember) != 0;
    if (!bad && orc_work_alloc(&wk, orc_max_degree(n, off)) != 0) bad = 1;
    if (bad) {
        free(first);
        free(member);
        free(tfirst);
        free(tmember);
        free(newc);
        free(taken);
        return -1;
    }
    for (int l = start_iter; l < max_iters; ++l) {
        int pl = (pl_period > 0) && (l % pl_period == 0);
        int64_t changed = 0, scanned = 0;
        for (int32_t q = 0; q < n_waves; ++q) {
            /* the wave starts: flags taken (each vertex marks itself processed) */
            for (int64_t r = tfirst[q]; r < tfirst[q + 1]; ++r) {
                const int64_t i = tmember[r];
                taken[i] = active[i];
                active[i] = 0;
            }
            /* the wave reads: c* of every deciding vertex whose flag was set, on the labels at its start */
            for (int64_t r = first[q]; r < first[q + 1]; ++r) {
                const int64_t i = member[r];
                newc[i] = -1;
                if (!taken[i]) continue;
                scanned += off[i + 1] - off[i];
                newc[i] = orc_best_label(i, off, idx, w, C, wk.lab, wk.sum, wk.scratch);
            }
            /* the wave writes: moves and neighbour marks */
            for (int64_t r = first[q]; r < first[q + 1]; ++r) {
                const int64_t i = member[r];
                const int32_t c = newc[i];
                if (c < 0) continue;
                const int32_t cur = C[i];
                if (c != cur && (!pl || c < cur)) {
                    C[i] = c;
                    ++changed;
                    for (int64_t e = off[i]; e < off[i + 1]; ++e) active[idx[e]] = 1;
                }
            }
        }
        dN[l] = changed;
        if (edges) edges[l] = scanned;
        *iters = l + 1;
        if (!pl && (double)changed / (double)n < tol) {
            *converged = 1;
            break;
        }
    }
    free(first);
    free(member);
    free(tfirst);
    free(tmember);
    free(newc);
    free(taken);
    orc_work_free(&wk);
    return 0;
}

/* One synchronous sweep over vertices [v0, v1) only, with all of them active and the
 * given frozen labels C (all n labels): the per-vertex step of Algorithm 1 (lpaMove) on a
 * bounded sample.  The rows come as a window: off_w[k] - off_w[0] is where row v0+k starts
 * in idx_w / w_w (length v1 - v0 + 1).  Writes the new labels of [v0, v1) to out and
 * returns the number of CSR entries scanned, or -1 on allocation failure. */
int64_t orc_sweep_window(int64_t v0, int64_t v1, const int64_t *off_w, const int32_t *idx_w,
                         const float *w_w, const int32_t *C, int pl, int32_t *out)
{
    const int64_t nv = v1 - v0, base = off_w[0];
    int64_t dmax = 0;
    for (int64_t k = 0; k < nv; ++k)
        if (off_w[k + 1] - off_w[k] > dmax) dmax = off_w[k + 1] - off_w[k];
    /* a one-row CSR per vertex: offsets {0, D}, rows taken from the window */
    orc_work wk;
    if (orc_work_alloc(&wk, dmax) != 0) return -1;
    for (int64_t k = 0; k < nv; ++k) {
        const int64_t i = v0 + k;
        const int64_t b = off_w[k] - base, d = off_w[k + 1] - off_w[k];
        int64_t cnt = 0;
        for (int64_t e = 0; e < d; ++e) {
            const int32_t j = idx_w[b + e];
            if (j == i) continue;
            wk.scratch[cnt].label = C[j];
            wk.scratch[cnt].pos = e;
            wk.scratch[cnt].w = w_w ? w_w[b + e] : 1.0f;
            ++cnt;
        }
        qsort(wk.scratch, (size_t)cnt, sizeof(orc_item), orc_item_cmp);
        int32_t best = -1;
        float bw = 0.0f;
        for (int64_t q = 0; q < cnt;) {             /* sort-and-count, labels ascending */
            int32_t lab = wk.scratch[q].label;
            float sum = 0.0f;
            for (; q < cnt && wk.scratch[q].label == lab; ++q) sum += wk.scratch[q].w;
            if (best < 0 || sum > bw) {
                best = lab;
                bw = sum;
            }
        }
        const int32_t cur = C[i];
        out[k] = (best >= 0 && best != cur && (!pl || best < cur)) ? best : cur;
    }
    orc_work_free(&wk);
    return off_w[nv] - base;
}

/* Same on a whole CSR (offsets absolute). */
int64_t orc_sweep_range(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                        int pl, int64_t v0, int64_t v1, const int32_t *C, int32_t *out)
{
    (void)n;
    return orc_sweep_window(v0, v1, off + v0, idx + off[v0], w ? w + off[v0] : NULL, C, pl, out);
}

/* ---------------------------------------------------------------------------
 * Per-vertex open-addressing hashtable of Section 4.2 with the hybrid
 * quadratic-double probe of Algorithm 2, single-threaded ("not shared") form.
 *
 * Readings: capacity p1 = nextPow2(D) - 1 with nextPow2 the smallest power of two
 * strictly above D, so p1 is the smallest 2^k - 1 >= D; secondary modulus
 * p2 = 2*p1 + 1 (> p1 and coprime with it).  The probe keeps i and delta reduced mod
 * p1, which leaves the slot sequence s_t = i_t mod p1 unchanged (the recurrence is
 * linear).  Accumulation adds v (H_v[s] += v).  After max_retries probes a linear
 * scan from the last probed slot inserts the key (counted in *fallbacks).
 */
uint32_t orc_ht_capacity(int64_t degree)
{
    uint32_t p = 1;
    while ((int64_t)p < degree) p = 2 * p + 1;
    return p;                       /* 1, 3, 7, 15, ... */
}

int orc_ht_accumulate(int32_t *Hk, float *Hv, uint32_t p1, uint32_t p2, int32_t k, float v,
                      int max_retries, int64_t *fallbacks)
{
    uint64_t i = (uint64_t)k % p1;
    uint64_t delta = 1 % p1;
    uint64_t step2 = (uint64_t)k % p2;
    uint64_t s = i;
    for (int t = 0; t < max_retries; ++t) {
        s = i;                                           /* 1st hash: s = i mod p1 */
        if (Hk[s] == k || Hk[s] == ORC_EMPTY) {
            Hk[s] = k;
            Hv[s] += v;
            return 0;
        }
        i = (i + delta) % p1;
        delta = (2 * delta + step2) % p1;                /* 2nd hash: k mod p2 */
    }
    if (fallbacks) ++*fallbacks;
    for (uint32_t u = 1; u <= p1; ++u) {
        uint64_t q = (s + u) % p1;
        if (Hk[q] == k || Hk[q] == ORC_EMPTY) {
            Hk[q] = k;
            Hv[q] += v;
            return 1;
        }
    }
    return -1;                                           /* failed: table full */
}

/* Slot visited at probe t for key k (t < max_retries), for checking the reduced
 * recurrence against the unreduced one. */
uint32_t orc_ht_probe_slot(uint32_t p1, uint32_t p2, int32_t k, int t)
{
    uint64_t i = (uint64_t)k % p1, delta = 1 % p1, step2 = (uint64_t)k % p2;
    for (int r = 0; r < t; ++r) {
        i = (i + delta) % p1;
        delta = (2 * delta + step2) % p1;
    }
    return (uint32_t)i;
}

/* Builds the table of a multiset of (key, value) pairs inserted in order: clear,
 * accumulate each pair.  Hk/Hv hold p1 slots.  Returns 0, or -1 if an insert failed. */
int orc_ht_build(int64_t count, const int32_t *keys, const float *vals, uint32_t p1,
                 int max_retries, int32_t *Hk, float *Hv, int64_t *fallbacks)
{
    uint32_t p2 = 2 * p1 + 1;
    for (uint32_t s = 0; s < p1; ++s) {
        Hk[s] = ORC_EMPTY;
        Hv[s] = 0.0f;
    }
    for (int64_t q = 0; q < count; ++q)
        if (orc_ht_accumulate(Hk, Hv, p1, p2, keys[q], vals[q], max_retries, fallbacks) < 0) return -1;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Modularity, Eq. 1 in its community form: Q = sum_c [sigma_c/2m - (Sigma_c/2m)^2],
 * sigma_c = weight of CSR entries with both endpoints in c, Sigma_c = sum of K_i over
 * i in c, 2m = total CSR weight.  float64 throughout.  Labels must lie in [0, n).
 */
double orc_modularity(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                      const int32_t *C)
{
    double two_m = 0.0, sin = 0.0, sq = 0.0;
    double *Sig = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!Sig) return -2.0;
    for (int64_t i = 0; i < n; ++i) {
        double Ki = 0.0;
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            double we = w ? (double)w[e] : 1.0;
            Ki += we;
            if (C[idx[e]] == C[i]) sin += we;
        }
        two_m += Ki;
        Sig[C[i]] += Ki;
    }
    for (int64_t c = 0; c < n; ++c) sq += Sig[c] * Sig[c];
    free(Sig);
    if (two_m == 0.0) return 0.0;
    return sin / two_m - sq / (two_m * two_m);
}

/* Exact modularity for integer weights: Q = (2m*sum_c sigma_c - sum_c Sigma_c^2)/(2m)^2,
 * numerator and denominator as 128-bit integers split into (hi, lo) 64-bit halves.
 * Returns -1 if a weight is not an integer. */
int orc_modularity_exact(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                         const int32_t *C, int64_t *num_hi, uint64_t *num_lo,
                         int64_t *den_hi, uint64_t *den_lo)
{
    __int128 two_m = 0, sin = 0, sq = 0;
    __int128 *Sig = (__int128 *)calloc((size_t)(n > 0 ? n : 1), sizeof(__int128));
    if (!Sig) return -2;
    for (int64_t i = 0; i < n; ++i) {
        __int128 Ki = 0;
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            float wf = w ? w[e] : 1.0f;
            int64_t wi = (int64_t)wf;
            if ((float)wi != wf) {
                free(Sig);
                return -1;
            }
            Ki += wi;
            if (C[idx[e]] == C[i]) sin += wi;
        }
        two_m += Ki;
        Sig[C[i]] += Ki;
    }
    for (int64_t c = 0; c < n; ++c) sq += Sig[c] * Sig[c];
    free(Sig);
    __int128 num = two_m * sin - sq, den = two_m * two_m;
    *num_hi = (int64_t)(num >> 64);
    *num_lo = (uint64_t)num;
    *den_hi = (int64_t)(den >> 64);
    *den_lo = (uint64_t)den;
    return 0;
}

/* Vertices whose label is not a max-weight neighbour label: i with at least one
 * non-self neighbour and K_{i->C_i} < max_c K_{i->c} (any max label counts as valid). */
int64_t orc_violations(int64_t n, const int64_t *off, const int32_t *idx, const float *w,
                       const int32_t *C)
{
    orc_work wk;
    if (orc_work_alloc(&wk, orc_max_degree(n, off)) != 0) return -1;
    int64_t bad = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t nd = orc_label_weights(i, off, idx, w, C, wk.lab, wk.sum, wk.scratch);
        if (nd == 0) continue;
        float mx = 0.0f, own = 0.0f;
        for (int64_t k = 0; k < nd; ++k) {
            if (wk.sum[k] > mx) mx = wk.sum[k];
            if (wk.lab[k] == C[i]) own = wk.sum[k];
        }
        if (own < mx) ++bad;
    }
    orc_work_free(&wk);
    return bad;
}
