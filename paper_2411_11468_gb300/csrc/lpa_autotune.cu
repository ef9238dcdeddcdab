// Autotuning of the degree buckets: thresholds, lanes per group, block sizes and the hub
// chunk, picked by timing real runs.  Host code only; it drives the public entry points.
//
// The search is a coordinate descent over a fixed candidate list per parameter, started from
// the handle's current tuning: each candidate that passes the tuning checks is applied and
// timed on the caller's run (best of `reps` runs, CUDA events), and a candidate replaces the
// current tuning only when it is at least 2% faster.  Passes repeat until one changes nothing
// (at most three).  Tuning changes which kernel processes a vertex and the launch shapes, never
// the arithmetic or the tie-break, so the labels of a synchronous run do not depend on it.
#include <cfloat>
#include <cstring>
#include <vector>

#include "lpa_internal.h"

namespace {

struct Axis {
    void (*set)(lpa_tuning &, int);
    std::vector<int> values;
};

const std::vector<Axis> &axes()
{
    static const std::vector<Axis> a = {
        {[](lpa_tuning &t, int v) { t.hub_chunk = v; }, {4096, 8192, 16384, 32768}},
        {[](lpa_tuning &t, int v) { t.hub_cluster = v; }, {0, 1}},
        {[](lpa_tuning &t, int v) { t.cta_xl_threads = v; }, {512, 1024}},
        {[](lpa_tuning &t, int v) { t.cta_xl_max = v; }, {4095, 8191}},
        {[](lpa_tuning &t, int v) { t.cta_large_threads = v; }, {256, 512}},
        {[](lpa_tuning &t, int v) { t.cta_large_max = v; }, {2047, 4095}},
        {[](lpa_tuning &t, int v) { t.cta_threads = v; }, {64, 128, 256}},
        {[](lpa_tuning &t, int v) { t.cta_max = v; }, {511, 1023, 2047}},
        {[](lpa_tuning &t, int v) { t.warp_max = v; }, {127, 255, 511}},
        {[](lpa_tuning &t, int v) { t.group_max = v; }, {15, 31, 63}},
        {[](lpa_tuning &t, int v) { t.group_lanes = v; }, {4, 8, 16}},
        {[](lpa_tuning &t, int v) { t.thread_max = v; }, {3, 7}},
    };
    return a;
}

// Coordinate descent.  apply(t) installs a tuning (LPA_EINVAL: not applicable, skipped);
// time(&ms) measures the installed one.  On return the best tuning is installed.
template <class Apply, class Time>
int descend(const lpa_tuning &start, int reps, Apply apply, Time time, lpa_tuning *best, float *best_ms,
            int *evaluated)
{
    auto measure = [&](float *ms) {
        *ms = FLT_MAX;
        for (int r = 0; r < reps; ++r) {
            float x = 0.f;
            const int st = time(&x);
            if (st != LPA_OK) return st;
            if (x < *ms) *ms = x;
        }
        return LPA_OK;
    };
    lpa_tuning cur = start;
    float cur_ms = 0.f;
    int count = 0;
    LPA_CHECK(apply(cur));
    LPA_CHECK(measure(&cur_ms));
    ++count;
    for (int pass = 0; pass < 3; ++pass) {
        bool changed = false;
        for (const Axis &ax : axes()) {
            for (int v : ax.values) {
                lpa_tuning t = cur;
                ax.set(t, v);
                if (std::memcmp(&t, &cur, sizeof t) == 0) continue;
                const int st = apply(t);
                if (st == LPA_EINVAL) continue;
                if (st != LPA_OK) return st;
                float ms = 0.f;
                LPA_CHECK(measure(&ms));
                ++count;
                if (ms < 0.98f * cur_ms) {
                    cur = t;
                    cur_ms = ms;
                    changed = true;
                }
            }
        }
        if (!changed) break;
    }
    LPA_CHECK(apply(cur));
    if (best) *best = cur;
    if (best_ms) *best_ms = cur_ms;
    if (evaluated) *evaluated = count;
    return LPA_OK;
}

bool run_args_ok(int max_iters, int pl_period, int mode, int reps)
{
    return max_iters >= 1 && pl_period >= 0 && (mode == LPA_SYNC || mode == LPA_ASYNC) && reps >= 1 && reps <= 16;
}

}  // namespace

extern "C" {

int lpa_autotune(lpa_graph *g, double tolerance, int max_iters, int pl_period, int mode, int reps, lpa_tuning *best,
                 float *best_ms, int *evaluated)
{
    if (!g || !run_args_ok(max_iters, pl_period, mode, reps)) {
        lpa::set_error("lpa_autotune: bad arguments (max_iters >= 1, mode LPA_SYNC or LPA_ASYNC, 1 <= reps <= 16)");
        return LPA_EINVAL;
    }
    lpa_tuning start{};
    LPA_CHECK(lpa_get_tuning(g, &start));
    lpa_stats st{};
    auto apply = [&](const lpa_tuning &t) { return lpa_set_tuning(g, &t); };
    auto time = [&](float *ms) {
        st.time_kernels = 0;
        LPA_CHECK(lpa_run(g, tolerance, max_iters, pl_period, mode, &st));
        *ms = st.total_ms;
        return LPA_OK;
    };
    return descend(start, reps, apply, time, best, best_ms, evaluated);
}

int lpa_batch_autotune(lpa_batch *b, double tolerance, int max_iters, int pl_period, int mode, int reps,
                       lpa_tuning *best, float *best_ms, int *evaluated)
{
    if (!b || !run_args_ok(max_iters, pl_period, mode, reps)) {
        lpa::set_error("lpa_batch_autotune: bad arguments (max_iters >= 1, mode LPA_SYNC or LPA_ASYNC, 1 <= reps <= 16)");
        return LPA_EINVAL;
    }
    lpa_tuning start{};
    LPA_CHECK(lpa_batch_get_tuning(b, &start));
    auto apply = [&](const lpa_tuning &t) {
        const int st = lpa_batch_set_tuning(b, &t);
        if (st != LPA_OK) return st;
        float ms = 0.f;    // the first run after a change records the sweep graph: not timed
        return lpa_batch_run(b, tolerance, max_iters, pl_period, mode, nullptr, &ms);
    };
    auto time = [&](float *ms) { return lpa_batch_run(b, tolerance, max_iters, pl_period, mode, nullptr, ms); };
    return descend(start, reps, apply, time, best, best_ms, evaluated);
}

}  // extern "C"
