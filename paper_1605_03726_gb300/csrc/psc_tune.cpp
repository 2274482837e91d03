// psc_tune.cpp -- launch autotuner of a lattice.
//
// Every option it touches (persistent stretches, molecules per thread, block
// shape of the per-event kernels, Morton re-sort period) changes only how the
// work is scheduled on the GPU, never which molecule moves where: the claim
// rule resolves each event from the snapshot and the lowest id, whatever the
// launch shape or list order.  So the trials run real events of the
// simulation -- nothing is thrown away -- and the lattice ends exactly where
// an untuned run of the same number of events ends.
#include "psc.h"
#include "psc_internal.h"
#include "psc_runtime.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

using namespace psc;
using namespace psc_rt;

namespace {

struct Trial {
    int32_t persistent, run_per_thread, block_threads, blocks_per_sm, resort_period, tiles, graph_events;
};

void apply(psc_lattice* L, const Trial& t)
{
    graph_cache_clear(L);
    L->opt.persistent = t.persistent;
    L->opt.run_per_thread = t.run_per_thread;
    L->opt.block_threads = t.block_threads;
    L->opt.blocks_per_sm = t.blocks_per_sm;
    L->opt.resort_period = t.resort_period;
    L->opt.tiles = t.tiles;
    L->opt.graph_events = t.graph_events;
}

Trial current(const psc_lattice* L)
{
    return {L->opt.persistent, L->opt.run_per_thread, L->opt.block_threads, L->opt.blocks_per_sm,
            L->opt.resort_period, L->opt.tiles, L->opt.graph_events};
}

struct Timer {
    psc_lattice* L;
    int64_t budget;                 // events left
    int64_t ran = 0;
    int trials = 0;
    cudaEvent_t a = nullptr, b = nullptr;

    // run up to n events untimed
    int warm(int64_t n)
    {
        n = std::min(n, budget);
        if (n <= 0) return PSC_OK;
        const uint64_t e0 = L->events;
        int rc = drive(L, INFINITY, n);
        const int64_t done = (int64_t)(L->events - e0);
        ran += done;
        budget -= done;
        return rc;
    }

    // run n events timed on the lattice's stream; *us = microseconds per event
    int timed(int64_t n, double* us)
    {
        *us = INFINITY;
        n = std::min(n, budget);
        if (n <= 0) return PSC_OK;
        const uint64_t e0 = L->events;
        if (cudaEventRecord(a, L->stream) != cudaSuccess) return PSC_E_CUDA;
        int rc = drive(L, INFINITY, n);
        if (cudaEventRecord(b, L->stream) != cudaSuccess) return PSC_E_CUDA;
        if (rc) return rc;
        if ((rc = check_device(L))) return rc;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return PSC_E_CUDA;
        const int64_t done = (int64_t)(L->events - e0);
        ran += done;
        budget -= done;
        ++trials;
        if (done > 0) *us = 1e3 * (double)ms / (double)done;
        return PSC_OK;
    }
};

// lists start every re-sort trial freshly sorted, as they do after a re-sort
int resort_all(psc_lattice* L)
{
    for (int s = 0; s < L->nsp; ++s) {
        if (!(L->sp[s].D > 0.0)) continue;
        int rc = resort(L, s);
        if (rc) return rc;
        L->since_resort[s] = 0;
    }
    return PSC_OK;
}

}  // namespace

extern "C" int psc_autotune(psc_lattice* L, int64_t max_events, psc_tune_result* out)
{
    if (!L || !out || max_events < 0) return PSC_E_ARG;
    std::memset(out, 0, sizeof(*out));
    if (!L->populated) return PSC_E_ORDER;
    if (L->sticky) return L->sticky;
    DevGuard dg(L->device);
    Timer T{L, max_events};
    if (cudaEventCreate(&T.a) != cudaSuccess || cudaEventCreate(&T.b) != cudaSuccess) {
        if (T.a) cudaEventDestroy(T.a);
        return PSC_E_CUDA;
    }
    const int saved_timing = L->opt.time_kernels;
    L->opt.time_kernels = 0;

    bool any_mobile = false, any_run = false;
    for (int s = 0; s < L->nsp; ++s) {
        if (!(L->sp[s].D > 0.0)) continue;
        any_mobile = true;
        if (!L->general[s]) any_run = true;
    }
    // about 17 trials of a window each, plus the re-sort trials' longer windows
    const int64_t W = std::max<int64_t>(4, std::min<int64_t>(256, max_events / 32));
    int rc = PSC_OK;
    Trial best = current(L);
    double best_us = INFINITY;
    auto run_trial = [&](const Trial& t, int64_t window, bool sorted_start, double* us) -> int {
        apply(L, t);
        int r = T.warm(2);                   // first launches of a new shape set kernel attributes
        if (r) return r;
        if (sorted_start && (r = resort_all(L))) return r;
        return T.timed(window, us);
    };

    if (any_mobile) {
        // the configuration in force: the reference point
        rc = run_trial(best, W, false, &best_us);
        out->us_per_event_before = best_us;

        // 1. block shape of the per-event kernels (every species that is not
        //    in a persistent stretch, and all species when stretches are off)
        const int32_t threads[] = {128, 256};
        const int32_t per_sm[] = {4, 8, 16};
        for (int32_t th : threads) {
            for (int32_t bp : per_sm) {
                if (rc || T.budget <= 0) break;
                Trial t = best;
                t.block_threads = th;
                t.blocks_per_sm = bp;
                if (t.block_threads == best.block_threads && t.blocks_per_sm == best.blocks_per_sm) continue;
                double us;
                rc = run_trial(t, W, false, &us);
                if (!rc && us < best_us) { best = t; best_us = us; }
            }
        }
        // 2. persistent stretches: the tile kernel, or molecules per thread of
        //    the molecule-list kernel, or none
        if (any_run) {
            const Trial cand[] = {{1, 0, 0, 0, 0, 1, 0}, {1, 0, 0, 0, 0, -1, 0}, {1, 8, 0, 0, 0, -1, 0},
                                  {1, 16, 0, 0, 0, -1, 0}, {-1, 0, 0, 0, 0, -1, 0}};
            for (const Trial& c : cand) {
                if (rc || T.budget <= 0) break;
                Trial t = best;
                t.persistent = c.persistent;
                t.run_per_thread = c.run_per_thread;
                t.tiles = c.tiles;
                if ((t.persistent > 0) == (best.persistent > 0) && t.run_per_thread == best.run_per_thread &&
                    t.tiles == best.tiles)
                    continue;
                double us;
                rc = run_trial(t, W, false, &us);
                if (!rc && us < best_us) { best = t; best_us = us; }
            }
        }
        // 3. re-sort period: each trial starts from sorted lists and spans at
        //    least two periods, so the re-sort cost is amortised as in a run
        const int32_t periods[] = {16, 32, 64, 128, 256, 512, -1};
        double p_best_us = INFINITY;
        Trial p_best = best;
        for (int32_t P : periods) {
            if (rc || T.budget <= 0) break;
            const int64_t window = P > 0 ? std::max<int64_t>(W, 2 * (int64_t)P) : std::max<int64_t>(W, 512);
            if (window > T.budget) continue;
            Trial t = best;
            t.resort_period = P;
            double us;
            rc = run_trial(t, window, true, &us);
            if (!rc && us < p_best_us) { p_best = t; p_best_us = us; }
        }
        if (!rc && p_best_us < INFINITY) { best = p_best; best_us = p_best_us; }
        // 4. graph replay of per-event runs, where events take per-event
        //    launches (species with reactions, or stretches off): a trial
        //    first runs three runs' worth of events, so that its patterns are
        //    seen and captured, then times a window of at least two runs
        bool per_event = best.persistent <= 0;
        for (int s = 0; s < L->nsp; ++s)
            if (L->sp[s].D > 0.0 && L->general[s]) per_event = true;
        if (per_event) {
            const int32_t ks[] = {0, 32, 128};
            double g_best_us = INFINITY;
            Trial g_best = best;
            for (int32_t k : ks) {
                if (rc || T.budget <= 0) break;
                const int64_t warm = 3 * (int64_t)std::max<int32_t>(k, 1);
                const int64_t window = std::max<int64_t>(W, 2 * (int64_t)k);
                if (warm + window > T.budget) continue;
                Trial t = best;
                t.graph_events = k;
                apply(L, t);
                if ((rc = T.warm(warm))) break;
                double us;
                rc = T.timed(window, &us);
                if (!rc && us < g_best_us) { g_best = t; g_best_us = us; }
            }
            if (!rc && g_best_us < INFINITY) { best = g_best; best_us = g_best_us; }
        }
    }
    apply(L, best);
    L->opt.time_kernels = saved_timing;
    cudaEventDestroy(T.a);
    cudaEventDestroy(T.b);
    out->persistent = best.persistent;
    out->run_per_thread = best.run_per_thread;
    out->block_threads = best.block_threads;
    out->blocks_per_sm = best.blocks_per_sm;
    out->resort_period = best.resort_period;
    out->tiles = best.tiles;
    out->graph_events = best.graph_events;
    out->trials = T.trials;
    out->events = T.ran;
    out->us_per_event = best_us;
    return rc;
}
