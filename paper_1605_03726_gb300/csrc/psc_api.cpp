// psc_api.cpp -- host runtime of the hop engine: the C ABI of include/psc.h.
//
// The host owns the model (species, reactions), derives the per-species
// constants of the paper (hop interval, Sec. 2.3; acceptance p_AB,
// Sec. 2.4.2; first-order firing, Sec. 2.4.1), runs the event scheduler
// (Sec. 2.2) and queues the kernels of each event on the lattice's stream.
// No step of an event runs on the host: the kernels read the molecule counts
// from device memory, so the host never waits for the device between events.
#include "psc.h"
#include "psc_internal.h"
#include "psc_readout.h"
#include "psc_runtime.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

using namespace psc;

namespace {

psc_alloc_fn g_alloc = nullptr;
psc_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;
std::mutex g_alloc_mu;

// floor(min(p, 1) * 2^32): a 32-bit uniform u passes with probability p iff u < T
uint64_t prob_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 1ull << 32;
    return (uint64_t)std::floor(p * 4294967296.0);
}

// Sec. 2.3, Eq. 3: mean time to hop one voxel diameter, tau_d = 2 r_v^2 / (3 D)
double hop_interval(double rv, double D) { return (2.0 * rv * rv) / (3.0 * D); }

// Sec. 2.4.2, Eq. 6: discrete Collins-Kimball acceptance of a collision
double acceptance(double k, double DA, double DB, double rv)
{
    return k / (6.0 * std::sqrt(2.0) * (DA + DB) * rv);
}

}  // namespace

namespace psc_rt {

int cuda_fail(psc_lattice* L, cudaError_t e)
{
    if (e == cudaSuccess) return PSC_OK;
    if (L) L->sticky = (e == cudaErrorMemoryAllocation) ? PSC_E_NOMEM : PSC_E_CUDA;
    return e == cudaErrorMemoryAllocation ? PSC_E_NOMEM : PSC_E_CUDA;
}

void* dev_alloc(psc_lattice* L, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        if (g_alloc) p = g_alloc(bytes, L->device, L->stream, g_alloc_ctx);
        else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    }
    if (p) L->allocs.push_back(p);
    return p;
}

void dev_free_all(psc_lattice* L)
{
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    for (void* p : L->allocs) {
        if (g_free) g_free(p, L->device, L->stream, g_alloc_ctx);
        else cudaFree(p);
    }
    L->allocs.clear();
}

void dev_free_one(psc_lattice* L, void* p)
{
    auto it = std::find(L->allocs.begin(), L->allocs.end(), p);
    if (it == L->allocs.end()) return;
    L->allocs.erase(it);
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_free) g_free(p, L->device, L->stream, g_alloc_ctx);
    else cudaFree(p);
}

int event_blocks(const psc_lattice* L, int64_t work)
{
    const int64_t want = (work + L->opt.block_threads - 1) / L->opt.block_threads;
    const int64_t cap = (int64_t)L->sm_count * L->opt.blocks_per_sm;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

// Grid of a per-event launch over list x: the list's grid class (4, 32 or
// 256 blocks, or the full grid for its capacity).
int list_blocks(const psc_lattice* L, int x)
{
    return std::min(event_blocks(L, L->cap[x]), L->grid_class[x]);
}

// The grid class for a list estimated at n entries, given its class so far:
// a class holds at least one block per 128 entries; it grows as soon as the
// list outgrows it and shrinks only once the list needs a sixteenth of it, so
// that captured graphs (keyed by the grids) stay valid while a count hovers.
static int grid_class_for(const psc_lattice* L, int x, int64_t n, int cur)
{
    static const int kClasses[3] = {4, 32, 256};
    const int full = event_blocks(L, L->cap[x]);
    const int64_t need = (2 * n + L->opt.block_threads - 1) / L->opt.block_threads + 1;
    int fit = INT32_MAX;
    for (int c : kClasses)
        if (need <= c && c < full) { fit = c; break; }
    if (cur <= 0 || fit > cur) return fit;                      // first class, or grown out of it
    const int64_t cur_blocks = std::min(cur, full);
    return need * 16 <= cur_blocks ? fit : cur;
}

// How many leading entries of list x a Morton re-sort takes: a list in a
// small grid class sorts twice what its class holds, at most its capacity
// (entries beyond keep their places; list order never changes results).  The
// sort's tiles and scans follow this bound, not the capacity, which for
// reaction products is the whole lattice.
int32_t sort_limit(const psc_lattice* L, int x)
{
    return (int32_t)std::min<int64_t>(L->cap[x], 256 * (int64_t)L->grid_class[x]);
}

// Does Morton order pay for list x?  Only if the list holds at least 1/256 of
// the voxels (by its estimate): sparser lists share too few cache lines
// between neighbours in any order, and their re-sorts cost more than they
// save.  A skipped re-sort changes no result.
bool sorted_order_pays(const psc_lattice* L, int x)
{
    return !L->counts_h || L->est[x] * 256 >= L->V;
}

// Take the last background copy of the list lengths if it has landed, and
// start the next one every 64 events.  The host queues events far faster than
// the device runs them; once a copy is 256 events old the host waits for it,
// so the estimates stay recent (the device still has that many queued).
void refresh_estimates(psc_lattice* L)
{
    if (!L->counts_h) return;
    if (L->counts_pending) {
        if (cudaEventQuery(L->counts_ev) != cudaSuccess) {
            if (L->g - L->counts_g < 256u) return;
            if (cudaEventSynchronize(L->counts_ev) != cudaSuccess) {
                L->counts_pending = false;
                return;
            }
        }
        for (int s = 0; s < L->nsp; ++s) {
            L->est[s] = L->counts_h[s];
            L->grid_class[s] = grid_class_for(L, s, L->est[s], L->grid_class[s]);
        }
        L->counts_pending = false;
    }
    if (L->g - L->counts_g < 64u) return;
    if (cudaMemcpyAsync(L->counts_h, L->sc->counts, sizeof(int32_t) * (size_t)L->nsp, cudaMemcpyDeviceToHost,
                        L->stream) != cudaSuccess ||
        cudaEventRecord(L->counts_ev, L->stream) != cudaSuccess)
        return;
    L->d2h += sizeof(int32_t) * (size_t)L->nsp;
    L->counts_pending = true;
    L->counts_g = L->g;
}

// set-up of one event of species s, everything passed by value
EventArgs event_args(const psc_lattice* L, int s)
{
    EventArgs a{};
    a.geo = L->geo;
    a.geo.slot_map = (uint32_t)(L->opt.slot_map - 1);
    a.occ = L->occ;
    a.bits = L->bits + (size_t)L->sp[s].comp * L->mirror_n;
    a.ct.direct = L->claim;
    if (L->tables[0]) {
        const int cur = (int)(L->g & 1u), other = cur ^ 1;
        a.ct.hash = L->tables[cur];
        a.ct.hash_bits = L->hash_bits[s];
        a.ct.clear = L->tables[other];
        a.ct.clear_n = L->table_used[other];
    }
    a.live = L->live[s] ? 1 : 0;
    a.list = L->model_h.lists[s];
    a.count = &L->sc->counts[s];
    a.model = L->model_d;
    a.sc = L->sc;
    a.births = L->births;
    a.births_cap = L->births_cap;
    a.key0 = (uint32_t)L->seed;
    a.key1 = (uint32_t)(L->seed >> 32);
    a.g = L->g;
    a.g_base = nullptr;
    if (L->capture_g0 >= 0) {                         // captured for replay: index relative to the run's first
        a.g = L->g - (uint32_t)L->capture_g0;
        a.g_base = &L->sc->g_base;
    }
    a.dirty[0] = L->dirty[0];
    a.dirty[1] = L->dirty[1];
    a.dirty_words = L->dirty_words;
    // the claim outcomes live in the scratch list's third array between claim
    // and commit, the due species' leavers in its first (its capacity is the
    // largest list's; the list passes that use it come after)
    a.dec = reinterpret_cast<uint8_t*>(L->tmp.img);
    a.leave = L->tmp.vox;
    a.holes = reinterpret_cast<int32_t*>(L->tmp.ids);
    a.surv = reinterpret_cast<int32_t*>(L->tmp.img);
    a.g_bump = nullptr;
    a.s = s;
    a.collect_stats = L->opt.collect_stats > 0 ? 1 : 0;
    return a;
}

enum SpanKind { kSpanClaim = 0, kSpanCommit, kSpanReconcile, kSpanResort, kSpanRun, kSpanTile, kSpanTileLean };

cudaEvent_t take_event(psc_lattice* L)
{
    if (!L->event_pool.empty()) {
        cudaEvent_t e = L->event_pool.back();
        L->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// open a span: returns its start event (recorded now) or null when timing is off
cudaEvent_t span_open(psc_lattice* L)
{
    if (L->opt.time_kernels <= 0) return nullptr;
    cudaEvent_t a = take_event(L);
    if (a) cudaEventRecord(a, L->stream);
    return a;
}

void span_close(psc_lattice* L, cudaEvent_t a, int kind, int64_t events = 1)
{
    if (!a) return;
    cudaEvent_t b = take_event(L);
    if (!b) { L->event_pool.push_back(a); return; }
    cudaEventRecord(b, L->stream);
    L->spans.push_back({a, b, kind, events});
}

int resort(psc_lattice* L, int s)
{
    const int blocks = list_blocks(L, s);
    const SpeciesList& list = L->model_h.lists[s];
    const int32_t* count = &L->sc->counts[s];
    const int32_t limit = sort_limit(L, s);
    launch_morton_keys(list, count, limit, L->geo, L->rs_keys, L->rs_vals, blocks, L->stream);
    if (radix_sort_pairs(L->rs_keys, L->rs_vals, count, limit, limit, (int)morton_sort_bits(L->geo),
                         L->rs_scratch, L->stream, &L->launches) != 0)
        return cuda_fail(L, cudaErrorUnknown);
    launch_permute(list, L->tmp, L->rs_vals, count, limit, blocks, L->stream);
    launch_copy_list(L->tmp, list, count, limit, blocks, L->stream);
    L->launches += 3;
    return PSC_OK;
}

ReconcileArgs reconcile_args(const psc_lattice* L, int x)
{
    ReconcileArgs r{};
    r.geo = L->geo;
    r.occ = L->occ;
    r.bits = L->bits + (size_t)L->sp[x].comp * L->mirror_n;
    r.x = x;
    r.list = L->model_h.lists[x];
    r.tmp = L->tmp;
    r.model = L->model_d;
    r.sc = L->sc;
    r.dirty[0] = L->dirty[0];
    r.dirty[1] = L->dirty[1];
    r.g = L->g;
    r.g_base = nullptr;
    r.g_bump = nullptr;
    if (L->capture_g0 >= 0) {
        r.g = L->g - (uint32_t)L->capture_g0;
        r.g_base = &L->sc->g_base;
    }
    return r;
}

int enqueue_event(psc_lattice* L, int s)
{
    const EventArgs a = event_args(L, s);
    const int threads = L->opt.block_threads;
    const int blocks = list_blocks(L, s);
    // captured as a single-event graph: the event's last launch advances the
    // device's event index to the next event
    uint32_t* bump = L->capture_single ? &L->sc->g_base : nullptr;
    const std::vector<int>& Q = L->reconcile[s];
    // a list of at most a few hundred molecules: claim, commit and its own
    // fill in one block, one launch
    const bool one = L->general[s] && L->grid_class[s] <= 4;
    cudaEvent_t sp = span_open(L);
    if (one) {
        EventArgs a1 = a;
        if (!L->fo2[s] && Q.size() == 1) a1.g_bump = bump;
        launch_event_one(a1, L->stream);
        span_close(L, sp, kSpanClaim);
        L->launches += 1;
    } else {
        launch_claim(a, L->general[s], blocks, threads, L->stream);
        span_close(L, sp, kSpanClaim);
        sp = span_open(L);
        launch_commit(a, L->general[s], blocks, threads, L->stream);
        span_close(L, sp, kSpanCommit);
        L->launches += 2;
    }
    if (L->tables[0]) {
        const int cur = (int)(L->g & 1u);
        L->table_used[cur] = 1u << L->hash_bits[s];
        L->table_used[cur ^ 1] = 0;
    }
    sp = (!L->reconcile[s].empty() || L->fo2[s]) ? span_open(L) : nullptr;
    // the due species' own list changes only through its own molecules, whose
    // commit noted the leavers; partner lists are checked against the grid,
    // one after the other; then one launch fills every list (but the own one
    // of a one-block event), a block each (list order: the due species, then
    // the partners; each list's scratch range follows those of the lists
    // before it)
    uint32_t before = 0;
    for (int x : Q) {
        if (x != s) {
            launch_reconcile(reconcile_args(L, x), before, list_blocks(L, x), threads, L->stream);
            L->launches += 1;
        }
        before |= 1u << x;
    }
    if (Q.size() > (one ? 1u : 0u)) {
        ListFill f{};
        f.r = reconcile_args(L, s);
        before = 0;
        for (size_t q = 0; q < Q.size(); ++q) {
            if (one && Q[q] == s) {
                before |= 1u << s;
                continue;
            }
            f.x[f.n] = Q[q];
            f.list[f.n] = L->model_h.lists[Q[q]];
            f.before[f.n] = before;
            before |= 1u << Q[q];
            if (++f.n == kListFillMax || q + 1 == Q.size()) {
                if (!L->fo2[s] && q + 1 == Q.size()) f.r.g_bump = bump;
                launch_fill(f, L->stream);
                L->launches += 1;
                f.n = 0;
            }
        }
    }
    if (L->fo2[s]) {
        EventArgs ab = a;
        ab.g_bump = bump;
        launch_births(ab, L->stream);
        L->launches += 1;
    }
    span_close(L, sp, kSpanReconcile);
    L->events++;
    if (L->opt.resort_period > 0 && ++L->since_resort[s] >= (uint64_t)L->opt.resort_period) {
        L->since_resort[s] = 0;
        if (sorted_order_pays(L, s)) {
            sp = span_open(L);
            int rc = resort(L, s);
            span_close(L, sp, kSpanResort);
            if (rc) return rc;
        }
    }
    return cuda_fail(L, cudaPeekAtLastError());
}

// Can a stretch of events of species s run in one persistent launch?
int run_width(const psc_lattice* L, int s, int* threads, int* blocks)
{
    if (L->opt.persistent <= 0 || L->general[s]) return 0;
    if (L->tables[0] && L->hash_bits[s] > 27) return 0;
    return run_capacity(L->cap[s], threads, blocks, L->sm_count, L->opt.run_per_thread);
}

int enqueue_run(psc_lattice* L, int s, int n_events, int per_thread, int threads, int blocks)
{
    cudaStream_t st = L->stream;
    // both claim tables must start empty
    for (int t = 0; t < 2; ++t) {
        if (L->tables[t] && L->table_used[t]) {
            launch_fill_u64(L->tables[t], kEmptySlot, L->table_used[t], L->sm_count * 4, st);
            L->table_used[t] = 0;
            L->launches += 1;
        }
    }
    RunArgs r{};
    r.ev = event_args(L, s);
    r.tables[0] = L->tables[0];
    r.tables[1] = L->tables[1];
    r.n_events = n_events;
    r.barrier = L->barrier;
    r.barrier_timeout_ns = (uint64_t)L->opt.barrier_timeout_us * 1000ull;
    r.barrier_phantom = (uint32_t)L->opt.barrier_phantom;
    int rc = cuda_fail(L, cudaMemsetAsync(L->barrier, 0, sizeof(BarrierState), st));
    if (rc) return rc;
    cudaEvent_t sp = span_open(L);
    rc = cuda_fail(L, launch_run(r, blocks, threads, per_thread, st));
    span_close(L, sp, kSpanRun, n_events);
    if (rc) return rc;
    L->launches += 1;
    L->events += (uint64_t)n_events;
    return PSC_OK;
}

// ---------------------------------------------------------------------------
// tile kernel (owner-computes stretches)
// ---------------------------------------------------------------------------
// Does the plan spread the species' molecules evenly enough over the boxes?
// Every event waits for the fullest box, so the tile kernel's time grows with
// max / mean of the box loads, while the molecule-list kernel is balanced by
// construction and takes about 1.4 times the tile kernel's time on evenly
// spread molecules (measured at 512^3).  Decided once per species, from the
// loads at its first stretch (one count kernel and one small read-back);
// molecules confined to part of the lattice (a compartment, a cluster) pick
// the molecule-list kernel.
static bool tile_balanced(psc_lattice* L, int s, const TilePlan& P)
{
    const int64_t n = L->sp[s].n0;
    if (n <= 0 || P.regions <= 0) return false;
    int32_t* counts = (int32_t*)dev_alloc(L, (size_t)P.regions * 4);
    if (!counts) return false;
    TileArgs A{};
    A.ev = event_args(L, s);
    A.plan = P;
    std::vector<int32_t> h((size_t)P.regions, 0);
    bool ok = cudaMemsetAsync(counts, 0, (size_t)P.regions * 4, L->stream) == cudaSuccess;
    if (ok) {
        launch_tile_count(A, counts, std::max(1, std::min(2 * L->sm_count, (int)((n + 4095) / 4096))), L->stream);
        L->launches += 1;
        ok = cudaMemcpyAsync(h.data(), counts, (size_t)P.regions * 4, cudaMemcpyDeviceToHost, L->stream) ==
                 cudaSuccess &&
             cudaStreamSynchronize(L->stream) == cudaSuccess;
        L->d2h += (uint64_t)P.regions * 4;
    }
    dev_free_one(L, counts);
    if (!ok) return false;
    const int32_t mx = *std::max_element(h.begin(), h.end());
    return (double)mx * P.regions <= kTileMaxImbalance * (double)n;
}

bool tile_plan(psc_lattice* L, int s, TilePlan* P)
{
    if (L->opt.tiles < 0 || L->general[s] || L->live[s] || !(L->sp[s].D > 0.0)) return false;
    // automatic choice: the tile kernel wins from about 2^18 molecules on
    // lattices whose claims go to hash tables; on lattices of up to 2^22
    // voxels the molecule-list kernel's per-voxel claim words stay in L2 and
    // it wins at every density (measured on 128^3, 256^3 and 512^3)
    if (L->opt.tiles == 0 && (L->sp[s].n0 < ((int64_t)1 << 18) || L->V <= ((int64_t)1 << 22))) return false;
    if (L->sp[s].n0 <= 0) return false;
    // periodic axes must wrap whole bricks
    if ((L->bflags & PSC_PERIODIC_I) && (L->ni & 3)) return false;
    if ((L->bflags & PSC_PERIODIC_J) && (L->nj & 3)) return false;
    if ((L->bflags & PSC_PERIODIC_K) && (L->nk & 1)) return false;
    if (L->tile_smem < 0) L->tile_smem = tile_smem_limit(L->device);
    const int nbi = (L->ni + 3) / 4, nbj = (L->nj + 3) / 4, nbk = (L->nk + 1) / 2;
    int S = kTileBlocksPerSM * L->sm_count;
    if (L->opt.tile_regions > 0) S = std::min(S, L->opt.tile_regions);
    // the cut that minimises the largest box (work of the slowest block), then
    // the halo
    int64_t best_work = -1, best_box = 0;
    TilePlan best{};
    // owner tables, neighbourhood masks, outbox
    const int fcc = (L->bflags & PSC_FCC) ? 1 : 0;
    const int64_t owners = ((nbi + nbj + nbk + 15) & ~15) + (fcc ? 96 : 32) * 8 * 4 + kTileOutbox * 12 +
                           kTileQueue * 4;
    for (int pi = 1; pi <= std::min(std::min(nbi, S), 255); ++pi) {
        for (int pj = 1; pj <= std::min(std::min(nbj, S / pi), 255); ++pj) {
            for (int pk = 1; pk <= std::min(std::min(nbk, S / (pi * pj)), 255); ++pk) {
                const int ei = (nbi + pi - 1) / pi, ej = (nbj + pj - 1) / pj, ek = (nbk + pk - 1) / pk;
                const int64_t box = (int64_t)(ei + 2) * (ej + 2) * (ek + 2);
                if (((box + 3) & ~3) * 4 + owners > L->tile_smem) continue;
                if (ei > 512 || ej > 512 || ek > 512) continue;   // packed region coordinates
                const int64_t work = (int64_t)ei * ej * ek;
                if (best_work < 0 || work < best_work || (work == best_work && box < best_box)) {
                    best_work = work;
                    best_box = box;
                    best = TilePlan{pi, pj, pk, nbi, nbj, nbk, ei, ej, ek, pi * pj * pk, (int32_t)box, 0, fcc};
                }
            }
        }
    }
    if (best_work < 0) return false;
    const double share = (double)best_work / ((double)nbi * nbj * nbk);
    const int64_t cap = std::min<int64_t>(best_work * 32, (int64_t)(2.0 * share * (double)L->sp[s].n0) + 8192);
    if (cap > INT32_MAX / 2) return false;
    best.cap = (int32_t)cap;
    // the lean variant: HCP, whole bricks on every axis (so reflective walls
    // fall on brick faces), boxes at least two bricks thick (neighbour waits),
    // two or more boxes along every periodic axis (no box wraps onto itself)
    {
        const bool whole = (L->ni % 4) == 0 && (L->nj % 4) == 0 && (L->nk % 2) == 0;
        const bool thick = nbi / best.pi >= 2 && nbj / best.pj >= 2 && nbk / best.pk >= 2;
        const bool wraps = (!(L->bflags & PSC_PERIODIC_I) || best.pi >= 2) &&
                           (!(L->bflags & PSC_PERIODIC_J) || best.pj >= 2) &&
                           (!(L->bflags & PSC_PERIODIC_K) || best.pk >= 2);
        best.lean = (!fcc && whole && thick && wraps && L->opt.tile_lean >= 0 &&
                     lean_smem_bytes(best) <= L->tile_smem) ? 1 : 0;
    }
    if (L->opt.tiles == 0) {
        if (L->tile_auto[s] == 0) L->tile_auto[s] = tile_balanced(L, s, best) ? 1 : -1;
        if (L->tile_auto[s] < 0) return false;
    }
    *P = best;
    return true;
}

static int tile_buffers(psc_lattice* L, const TilePlan& P, int64_t ids)
{
    auto& T = L->tile;
    const int64_t slots = (int64_t)P.regions * P.cap;
    if (slots > T.slots || P.regions > T.regions) {
        for (void* p : {(void*)T.b_vox[0], (void*)T.b_vox[1], (void*)T.b_ids[0], (void*)T.b_ids[1],
                        (void*)T.b_state, (void*)T.b_cnt, (void*)T.in_vox, (void*)T.in_ids, (void*)T.in_cnt,
                        (void*)T.claimed, (void*)T.done})
            if (p) dev_free_one(L, p);
        const int64_t ns = std::max(slots, T.slots);
        const int32_t nr = std::max(P.regions, T.regions);
        for (int x = 0; x < 2; ++x) {
            T.b_vox[x] = (int32_t*)dev_alloc(L, (size_t)ns * 4);
            T.b_ids[x] = (uint32_t*)dev_alloc(L, (size_t)ns * 4);
        }
        T.b_state = (uint32_t*)dev_alloc(L, (size_t)ns * 4);
        T.in_vox = (int32_t*)dev_alloc(L, (size_t)ns * 4);
        T.in_ids = (uint32_t*)dev_alloc(L, (size_t)ns * 4);
        T.b_cnt = (int32_t*)dev_alloc(L, (size_t)nr * 4);
        T.in_cnt = (int32_t*)dev_alloc(L, (size_t)nr * 4);
        T.claimed = (uint32_t*)dev_alloc(L, (size_t)nr * 4);
        T.done = (uint32_t*)dev_alloc(L, (size_t)nr * 4);
        T.slots = ns;
        T.regions = nr;
        if (!T.b_vox[0] || !T.b_vox[1] || !T.b_ids[0] || !T.b_ids[1] || !T.b_state || !T.in_vox || !T.in_ids ||
            !T.b_cnt || !T.in_cnt || !T.claimed || !T.done) {
            T.slots = 0;
            return PSC_E_NOMEM;
        }
    }
    if (!L->claim && !T.claim) {
        // contested targets are claimed in per-voxel words, free (all ones) between events
        T.claim = (uint32_t*)dev_alloc(L, (size_t)L->V * 4);
        if (!T.claim) return PSC_E_NOMEM;
        launch_fill_u32(T.claim, kNoClaim, (size_t)L->V, L->sm_count * 8, L->stream);
    }
    if (P.lean && (int64_t)P.regions * lean_halo_cap(P) > T.halo_entries) {
        if (T.halo_tab) dev_free_one(L, T.halo_tab);
        const int64_t ne = (int64_t)P.regions * lean_halo_cap(P);
        T.halo_tab = (uint2*)dev_alloc(L, (size_t)ne * sizeof(uint2));
        T.halo_entries = T.halo_tab ? ne : 0;
        if (!T.halo_tab) return PSC_E_NOMEM;
    }
    if (ids > T.ids) {
        if (T.img_id) dev_free_one(L, T.img_id);
        T.img_id = (uint64_t*)dev_alloc(L, (size_t)ids * 8);
        T.ids = T.img_id ? ids : 0;
        if (!T.img_id) return PSC_E_NOMEM;
    }
    return PSC_OK;
}

int enqueue_tiles(psc_lattice* L, int s, int64_t n_events, const TilePlan& P)
{
    cudaStream_t st = L->stream;
    int64_t id_lo = 0;
    for (int q = 0; q < s; ++q) id_lo += L->sp[q].n0;
    int rc = tile_buffers(L, P, L->sp[s].n0);
    if (rc) return rc;
    TileArgs A{};
    A.ev = event_args(L, s);
    A.ev.ct.hash = nullptr;
    A.ev.ct.clear = nullptr;
    A.ev.ct.clear_n = 0;
    A.claim = L->claim ? L->claim : L->tile.claim;
    A.claimed = L->tile.claimed;
    A.done = L->tile.done;
    // Neighbour waits instead of grid barriers need boxes at least two bricks
    // thick: then everything a phase reads from outside its box (halo bits,
    // arrivals, the claim words of targets next to it) is written only by
    // boxes adjacent to it, and all boxes touching one claim word are
    // adjacent to each other.
    A.nbr_sync = (P.nbi / P.pi >= 2 && P.nbj / P.pj >= 2 && P.nbk / P.pk >= 2) ? 1 : 0;
    A.plan = P;
    for (int x = 0; x < 2; ++x) {
        A.b_vox[x] = L->tile.b_vox[x];
        A.b_ids[x] = L->tile.b_ids[x];
    }
    A.b_state = L->tile.b_state;
    A.b_cnt = L->tile.b_cnt;
    A.in_vox = L->tile.in_vox;
    A.in_ids = L->tile.in_ids;
    A.in_cnt = L->tile.in_cnt;
    A.img_id = L->tile.img_id;
    A.halo_tab = L->tile.halo_tab;
    A.halo_cap = P.lean ? (int32_t)lean_halo_cap(P) : 0;
    A.id_lo = (uint32_t)id_lo;
    A.n_events = (int32_t)n_events;
    A.barrier = L->barrier;
    A.barrier_timeout_ns = (uint64_t)L->opt.barrier_timeout_us * 1000ull;
    A.barrier_phantom = (uint32_t)L->opt.barrier_phantom;
    if ((rc = cuda_fail(L, cudaMemsetAsync(L->tile.b_cnt, 0, (size_t)P.regions * 4, st)))) return rc;
    if ((rc = cuda_fail(L, cudaMemsetAsync(L->tile.in_cnt, 0, (size_t)P.regions * 4, st)))) return rc;
    if ((rc = cuda_fail(L, cudaMemsetAsync(L->tile.done, 0, (size_t)P.regions * 4, st)))) return rc;
    if ((rc = cuda_fail(L, cudaMemsetAsync(L->tile.claimed, 0, (size_t)P.regions * 4, st)))) return rc;
    if ((rc = cuda_fail(L, cudaMemsetAsync(L->barrier, 0, sizeof(BarrierState), st)))) return rc;
    cudaEvent_t sp = span_open(L);
    const int64_t n = L->sp[s].n0;
    const int sblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 8191) / 8192, 2 * L->sm_count));
    launch_tile_scatter(A, sblocks, st);
    rc = cuda_fail(L, launch_tile_run(A, st));
    if (!rc) launch_tile_gather(A, st);
    span_close(L, sp, P.lean ? kSpanTileLean : kSpanTile, n_events);
    if (rc) return rc;
    L->launches += 3;
    L->events += (uint64_t)n_events;
    return cuda_fail(L, cudaPeekAtLastError());
}

// the sub-volume rule: one cooperative launch over a stretch of events
int enqueue_subvol(psc_lattice* L, int s, int64_t n_events)
{
    cudaStream_t st = L->stream;
    SubvolArgs A{};
    A.ev = event_args(L, s);
    A.word = L->subvol.word;
    A.head = L->subvol.head;
    A.next = L->subvol.next;
    A.state = L->subvol.state;
    A.colour0 = L->subvol.colour0;
    A.lead = L->subvol.lead;
    A.lead_vox = L->subvol.lead_vox;
    A.counters = L->subvol.counters;
    A.n_events = (int32_t)n_events;
    A.barrier = L->barrier;
    A.barrier_timeout_ns = (uint64_t)L->opt.barrier_timeout_us * 1000ull;
    A.barrier_phantom = (uint32_t)L->opt.barrier_phantom;
    int rc = cuda_fail(L, cudaMemsetAsync(L->barrier, 0, sizeof(BarrierState), st));
    if (rc) return rc;
    if ((rc = cuda_fail(L, cudaMemsetAsync(L->subvol.counters, 0, 32 * sizeof(uint32_t), st)))) return rc;
    cudaEvent_t sp = span_open(L);
    rc = cuda_fail(L, launch_subvol(A, L->subvol.blocks, 256, st));
    span_close(L, sp, kSpanRun, n_events);
    if (rc) return rc;
    L->launches += 1;
    L->events += (uint64_t)n_events;
    return PSC_OK;
}

// Sec. 2.2: the next event belongs to the mobile species whose next diffusion
// time (events done + 1) * tau is earliest; ties go to the lower index.
bool next_event(const psc_lattice* L, int* s_out, double* t_out)
{
    int best = -1;
    double tb = 0.0;
    for (int s = 0; s < L->nsp; ++s) {
        if (!(L->sp[s].D > 0.0)) continue;
        const double t = (double)(L->sp[s].done + 1) * L->sp[s].tau;
        if (best < 0 || t < tb) { best = s; tb = t; }
    }
    *s_out = best;
    *t_out = tb;
    return best >= 0;
}

int check_device(psc_lattice* L)
{
    cudaError_t e = cudaStreamSynchronize(L->stream);
    if (e != cudaSuccess) return cuda_fail(L, e);
    if (!L->populated) return L->sticky;
    int32_t err = 0;
    e = cudaMemcpy(&err, &L->sc->err, sizeof(err), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(L, e);
    L->d2h += sizeof(err);
    if (err & kErrBarrierTimeout) L->sticky = PSC_E_TIMEOUT;
    else if (err) L->sticky = PSC_E_CAPACITY;
    return L->sticky;
}



}  // namespace psc_rt

using namespace psc_rt;

extern "C" {

const char* psc_status_string(int s)
{
    switch (s) {
    case PSC_OK: return "PSC_OK";
    case PSC_E_ARG: return "PSC_E_ARG";
    case PSC_E_DIMS: return "PSC_E_DIMS";
    case PSC_E_ORDER: return "PSC_E_ORDER";
    case PSC_E_FULL: return "PSC_E_FULL";
    case PSC_E_UNSUPPORTED: return "PSC_E_UNSUPPORTED";
    case PSC_E_NOMEM: return "PSC_E_NOMEM";
    case PSC_E_CUDA: return "PSC_E_CUDA";
    case PSC_E_TIMEOUT: return "PSC_E_TIMEOUT";
    case PSC_E_LIMIT: return "PSC_E_LIMIT";
    case PSC_E_CAPACITY: return "PSC_E_CAPACITY";
    case PSC_W_PCLAMP: return "PSC_W_PCLAMP";
    default: return "PSC_UNKNOWN";
    }
}

int psc_set_allocator(psc_alloc_fn alloc, psc_free_fn release, void* ctx)
{
    if ((alloc == nullptr) != (release == nullptr)) return PSC_E_ARG;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return PSC_OK;
}

int psc_lattice_create(psc_lattice** out, int32_t ni, int32_t nj, int32_t nk, double rv,
                       uint32_t bflags, int device, void* cuda_stream)
{
    if (!out) return PSC_E_ARG;
    *out = nullptr;
    if (!(rv > 0.0) || !std::isfinite(rv) || bflags > 15u || device < 0) return PSC_E_ARG;
    if (ni < 1 || nj < 1 || nk < 1) return PSC_E_DIMS;
    const int64_t V = (int64_t)ni * nj * nk;
    if (V >= (1ll << 31)) return PSC_E_DIMS;
    if ((bflags & PSC_PERIODIC_I) && ni < 3) return PSC_E_DIMS;
    if ((bflags & PSC_PERIODIC_J) && (nj < 4 || (nj & 1))) return PSC_E_DIMS;
    if (!(bflags & PSC_FCC) && (bflags & PSC_PERIODIC_K) && (nk < 4 || (nk & 1))) return PSC_E_DIMS;
    if ((bflags & PSC_FCC) && (bflags & PSC_PERIODIC_K) && (nk < 3 || nk % 3)) return PSC_E_DIMS;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) return PSC_E_CUDA;
    psc_lattice* L = new (std::nothrow) psc_lattice();
    if (!L) return PSC_E_NOMEM;
    L->ni = ni; L->nj = nj; L->nk = nk; L->V = V; L->rv = rv; L->bflags = bflags; L->device = device;
    std::memset(L->pair, -1, sizeof(L->pair));
    DevGuard dg(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete L; return PSC_E_CUDA; }
    L->sm_count = prop.multiProcessorCount;
    if (cuda_stream) {
        L->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess) { delete L; return PSC_E_CUDA; }
        L->own_stream = true;
    }
    L->geo.ni = ni; L->geo.nj = nj; L->geo.nk = nk; L->geo.bflags = bflags;
    L->geo.ninj = (uint32_t)ni * (uint32_t)nj;
    L->geo.div_ni = make_fastdiv((uint32_t)ni);
    L->geo.div_ninj = make_fastdiv(L->geo.ninj);
    L->geo.nbi = (uint32_t)((ni + 3) / 4);
    L->geo.nbj = (uint32_t)((nj + 3) / 4);
    *out = L;
    return PSC_OK;
}

int psc_add_species(psc_lattice* L, double D, int64_t n0, int32_t* species_out)
{
    if (!L) return PSC_E_ARG;
    if (L->populated) return PSC_E_ORDER;
    if (!(D >= 0.0) || !std::isfinite(D) || n0 < 0) return PSC_E_ARG;
    if (L->nsp >= kMaxSpecies) return PSC_E_UNSUPPORTED;
    Species& S = L->sp[L->nsp];
    S = Species();
    S.D = D;
    S.n0 = n0;
    S.tau = D > 0.0 ? hop_interval(L->rv, D) : 0.0;
    if (species_out) *species_out = L->nsp;
    L->nsp++;
    return PSC_OK;
}

int psc_add_reaction(psc_lattice* L, const int32_t* re, int32_t nr, const int32_t* pr, int32_t np,
                     double k, int32_t* rx_out)
{
    if (!L) return PSC_E_ARG;
    if (L->populated) return PSC_E_ORDER;
    if (nr < 1 || nr > 2 || np < 0 || !re || (np > 0 && !pr)) return PSC_E_ARG;
    if (!(k >= 0.0) || !std::isfinite(k)) return PSC_E_ARG;
    if (np > 2) return PSC_E_UNSUPPORTED;
    for (int a = 0; a < nr; ++a) if (re[a] < 0 || re[a] >= L->nsp) return PSC_E_ARG;
    for (int a = 0; a < np; ++a) if (pr[a] < 0 || pr[a] >= L->nsp) return PSC_E_ARG;
    if (L->nrx >= kMaxReactions) return PSC_E_UNSUPPORTED;
    if (nr == 2) {
        if (re[0] == re[1]) return PSC_E_UNSUPPORTED;
        if (!(L->sp[re[0]].D + L->sp[re[1]].D > 0.0)) return PSC_E_UNSUPPORTED;
        if (L->pair[re[0]][re[1]] >= 0) return PSC_E_UNSUPPORTED;
    } else {
        if (!(L->sp[re[0]].D > 0.0)) return PSC_E_UNSUPPORTED;
        if (L->sp[re[0]].n_fo >= kMaxFirstOrder) return PSC_E_UNSUPPORTED;
    }
    Reaction& R = L->rx[L->nrx];
    R = Reaction();
    R.nr = nr; R.np = np; R.k = k;
    for (int a = 0; a < nr; ++a) R.r[a] = re[a];
    for (int a = 0; a < np; ++a) R.p[a] = pr[a];
    if (nr == 2) {
        L->pair[re[0]][re[1]] = (int8_t)L->nrx;
        L->pair[re[1]][re[0]] = (int8_t)L->nrx;
    } else {
        Species& S = L->sp[re[0]];
        S.fo[S.n_fo++] = L->nrx;
    }
    if (rx_out) *rx_out = L->nrx;
    L->nrx++;
    return PSC_OK;
}

int psc_set_compartments(psc_lattice* L, const uint8_t* labels, int32_t n)
{
    if (!L || !labels) return PSC_E_ARG;
    if (L->populated) return PSC_E_ORDER;
    if (n < 1 || n > kMaxCompartments) return PSC_E_ARG;
    for (int64_t v = 0; v < L->V; ++v)
        if (labels[v] >= n) return PSC_E_ARG;
    for (int s = 0; s < L->nsp; ++s)
        if (L->sp[s].comp >= n) return PSC_E_ARG;
    L->labels.assign(labels, labels + L->V);
    L->ncomp = n;
    return PSC_OK;
}

int psc_species_compartment(psc_lattice* L, int32_t s, int32_t c)
{
    if (!L || s < 0 || s >= L->nsp) return PSC_E_ARG;
    if (L->populated) return PSC_E_ORDER;
    if (c < 0 || c >= L->ncomp) return PSC_E_ARG;
    L->sp[s].comp = c;
    return PSC_OK;
}

double psc_tau(const psc_lattice* L, int32_t s)
{
    if (!L || s < 0 || s >= L->nsp || !(L->sp[s].D > 0.0)) return 0.0;
    return L->sp[s].tau;
}

double psc_p_ab(const psc_lattice* L, int32_t r)
{
    if (!L || r < 0 || r >= L->nrx || L->rx[r].nr != 2) return 0.0;
    const Reaction& R = L->rx[r];
    return acceptance(R.k, L->sp[R.r[0]].D, L->sp[R.r[1]].D, L->rv);
}

int psc_populate(psc_lattice* L, uint64_t seed)
{
    if (!L) return PSC_E_ARG;
    if (L->populated) return PSC_E_ORDER;
    int64_t N = 0;
    for (int s = 0; s < L->nsp; ++s) N += L->sp[s].n0;
    if (N > L->V) return PSC_E_FULL;
    // compartments: room in each for its species, and products that can land
    // in theirs
    const bool comps = !L->labels.empty();
    int64_t start[kMaxSpecies] = {};                 // first sorted voxel of each species (placement)
    {
        int64_t room[kMaxCompartments] = {}, used[kMaxCompartments] = {};
        if (comps) {
            for (int64_t v = 0; v < L->V; ++v) room[L->labels[v]]++;
        } else {
            room[0] = L->V;
        }
        for (int s = 0; s < L->nsp; ++s) {
            const int c = L->sp[s].comp;
            used[c] += L->sp[s].n0;
            if (used[c] > room[c]) return PSC_E_FULL;
        }
        for (int r = 0; r < L->nrx; ++r) {
            const Reaction& R = L->rx[r];
            const int ca = L->sp[R.r[0]].comp;
            if (R.nr == 1) {
                if (R.np >= 1 && L->sp[R.p[0]].comp != ca) return PSC_E_UNSUPPORTED;
                continue;
            }
            const int cb = L->sp[R.r[1]].comp;
            if (R.np == 1 && L->sp[R.p[0]].comp != ca && L->sp[R.p[0]].comp != cb) return PSC_E_UNSUPPORTED;
            if (R.np == 2) {
                const int c0 = L->sp[R.p[0]].comp, c1 = L->sp[R.p[1]].comp;
                if (!((c0 == ca && c1 == cb) || (c0 == cb && c1 == ca))) return PSC_E_UNSUPPORTED;
            }
        }
    }
    DevGuard dg(L->device);
    L->seed = seed;

    // ---- frozen constants (Sec. 2.3, 2.4.1, 2.4.2) ----
    ModelDev& M = L->model_h;
    std::memset(&M, 0, sizeof(M));
    std::memcpy(M.pair, L->pair, sizeof(M.pair));
    bool growth = false;
    bool is_product[kMaxSpecies] = {};
    for (int r = 0; r < L->nrx; ++r) {
        Reaction& R = L->rx[r];
        ReactionDev& D = M.rx[r];
        D.np = R.np;
        D.p0 = R.np > 0 ? R.p[0] : 0;
        D.p1 = R.np > 1 ? R.p[1] : 0;
        for (int a = 0; a < R.np; ++a) is_product[R.p[a]] = true;
        if (R.nr == 2) {
            R.prob = acceptance(R.k, L->sp[R.r[0]].D, L->sp[R.r[1]].D, L->rv);
            if (R.prob > 1.0) L->clamped = true;
            D.T = prob_threshold(R.prob);
        } else if (R.np == 2) {
            growth = true;
        }
    }
    for (int s = 0; s < L->nsp; ++s) {
        const Species& S = L->sp[s];
        M.n_fo[s] = S.n_fo;
        if (S.n_fo == 0) continue;
        // per molecule and per own diffusion event: fire with 1 - exp(-a0 tau)
        double ktot = 0.0;
        for (int u = 0; u < S.n_fo; ++u) ktot += L->rx[S.fo[u]].k;
        M.T_fire[s] = prob_threshold(-std::expm1(-ktot * S.tau));
        // Eq. 5: reaction u is the first whose cumulative share reaches a0 R
        double cum = 0.0;
        for (int u = 0; u < S.n_fo; ++u) {
            cum += L->rx[S.fo[u]].k;
            M.fo_rx[s][u] = S.fo[u];
            M.fo_cum[s][u] = (u == S.n_fo - 1) ? (1ull << 32)
                                               : prob_threshold(ktot > 0.0 ? cum / ktot : 1.0);
        }
    }
    // ---- which lists an event can touch ----
    for (int s = 0; s < L->nsp; ++s) L->live[s] = false;
    for (int r = 0; r < L->nrx; ++r) {
        for (int a = 0; a < L->rx[r].nr; ++a) L->live[L->rx[r].r[a]] = true;
        for (int a = 0; a < L->rx[r].np; ++a) L->live[L->rx[r].p[a]] = true;
    }
    for (int s = 0; s < L->nsp; ++s) {
        bool so = false;
        L->reconcile[s].clear();
        for (int r = 0; r < L->nsp; ++r) if (L->pair[s][r] >= 0) so = true;
        L->general[s] = so || L->sp[s].n_fo > 0;
        L->fo2[s] = false;
        for (int u = 0; u < L->sp[s].n_fo; ++u)
            if (L->rx[L->sp[s].fo[u]].np == 2) L->fo2[s] = true;
        if (L->general[s]) {
            L->reconcile[s].push_back(s);
            for (int r = 0; r < L->nsp; ++r) if (L->pair[s][r] >= 0) L->reconcile[s].push_back(r);
        }
    }
    // ---- the sub-volume rule takes species without reactions on colour-consistent periods ----
    if (L->opt.subvolume > 0) {
        for (int s = 0; s < L->nsp; ++s)
            if (L->sp[s].D > 0.0 && L->general[s]) return PSC_E_UNSUPPORTED;
        if (((L->bflags & PSC_PERIODIC_I) && L->ni % 4) || ((L->bflags & PSC_PERIODIC_J) && L->nj % 4) ||
            ((L->bflags & PSC_PERIODIC_K) && L->nk % 4))
            return PSC_E_DIMS;
    }
    // ---- capacities: a list only grows if its species is a product ----
    const int64_t total_bound = growth ? L->V : N;
    int64_t max_cap = 1, max_mobile = 1;
    for (int s = 0; s < L->nsp; ++s) {
        int64_t c = is_product[s] ? std::min<int64_t>(L->V, std::max<int64_t>(total_bound, L->sp[s].n0))
                                  : L->sp[s].n0;
        c = std::max<int64_t>(c, 1);
        L->cap[s] = (int32_t)c;
        max_cap = std::max(max_cap, c);
        if (L->sp[s].D > 0.0) max_mobile = std::max(max_mobile, c);
    }
    bool any_fo2 = false;
    for (int s = 0; s < L->nsp; ++s) any_fo2 = any_fo2 || L->fo2[s];

    // ---- device memory ----
    const size_t V = (size_t)L->V;
    const size_t nwords = (size_t)mirror_words(L->ni, L->nj, L->nk);
    const int nmirror = comps ? L->ncomp : 1;
    L->mirror_n = nwords;
    L->occ = (uint16_t*)dev_alloc(L, V * sizeof(uint16_t));
    L->bits = (uint32_t*)dev_alloc(L, nwords * nmirror * sizeof(uint32_t));
    L->dirty_words = (uint32_t)((nwords + 31) / 32);
    for (int x = 0; x < 2; ++x) {
        L->dirty[x] = (uint32_t*)dev_alloc(L, (size_t)L->dirty_words * 4);
        if (!L->dirty[x]) return PSC_E_NOMEM;
    }
    L->sc = (Scalars*)dev_alloc(L, sizeof(Scalars));
    L->model_d = (ModelDev*)dev_alloc(L, sizeof(ModelDev));
    L->barrier = (BarrierState*)dev_alloc(L, sizeof(BarrierState));
    uint32_t* mort = (uint32_t*)dev_alloc(L, (size_t)(L->ni + L->nj + L->nk) * sizeof(uint32_t));
    if (!L->occ || !L->bits || !L->sc || !L->model_d || !L->barrier || !mort) return PSC_E_NOMEM;
    {
        std::vector<uint32_t> mt((size_t)(L->ni + L->nj + L->nk));
        uint32_t mbits = 0;
        build_morton_tables(L->ni, L->nj, L->nk, mt.data(), &mbits);
        int rc0 = cuda_fail(L, cudaMemcpy(mort, mt.data(), mt.size() * 4, cudaMemcpyHostToDevice));
        if (rc0) return rc0;
        L->h2d += mt.size() * 4;
        L->geo.mort = mort;
        L->geo.mort_bits = mbits;
    }
    // claims: a word per voxel on small lattices, else two hash tables with at
    // least two slots per molecule of the largest mobile species
    uint32_t hb_max = 0;
    for (int s = 0; s < L->nsp; ++s) {
        uint32_t hb = 10;
        while (hb < 31 && (1ll << hb) < (int64_t)L->opt.claim_slots * L->cap[s]) ++hb;
        L->hash_bits[s] = hb;
        if (L->sp[s].D > 0.0 && hb > hb_max) hb_max = hb;
    }
    bool direct = L->V <= (1ll << 22) || hb_max == 0;
    // tables at least as large as a word per voxel buy nothing, and the
    // per-event kernels empty the previous table in full every event (species
    // that are reaction products get lists sized for the lattice)
    if (2.0 * 8.0 * (double)(1ll << hb_max) >= 4.0 * (double)L->V) direct = true;
    if (L->opt.claim_table == 1) direct = true;
    if (L->opt.claim_table == 2 && hb_max > 0) direct = false;
    if (direct) {
        L->claim = (uint32_t*)dev_alloc(L, V * sizeof(uint32_t));
        if (!L->claim) return PSC_E_NOMEM;
    } else {
        L->table_slots = (int64_t)1 << hb_max;
        for (int t = 0; t < 2; ++t) {
            L->tables[t] = (uint64_t*)dev_alloc(L, ((size_t)1 << hb_max) * sizeof(uint64_t));
            if (!L->tables[t]) return PSC_E_NOMEM;
        }
    }
    for (int s = 0; s < L->nsp; ++s) {
        M.comp[s] = (uint8_t)(comps ? L->sp[s].comp : 0);
        M.mirror[s] = L->bits + (size_t)M.comp[s] * nwords;
        SpeciesList& l = M.lists[s];
        l.cap = L->cap[s];
        l.vox = (int32_t*)dev_alloc(L, (size_t)l.cap * 4);
        l.ids = (uint32_t*)dev_alloc(L, (size_t)l.cap * 4);
        l.img = (uint64_t*)dev_alloc(L, (size_t)l.cap * 8);
        if (!l.vox || !l.ids || !l.img) return PSC_E_NOMEM;
    }
    // the list passes of an event note up to two leavers per reaction, at most
    // one reaction per molecule of the due species
    L->tmp.cap = (int32_t)max_cap;
    L->tmp.vox = (int32_t*)dev_alloc(L, (size_t)max_cap * 8);
    L->tmp.ids = (uint32_t*)dev_alloc(L, (size_t)max_cap * 8);
    L->tmp.img = (uint64_t*)dev_alloc(L, (size_t)max_cap * 8);
    if (!L->tmp.vox || !L->tmp.ids || !L->tmp.img) return PSC_E_NOMEM;
    L->births_cap = any_fo2 ? 8192 : 1;
    L->births = (Birth*)dev_alloc(L, (size_t)L->births_cap * sizeof(Birth));
    L->rs_max = max_mobile;
    L->rs_keys = (uint32_t*)dev_alloc(L, (size_t)max_mobile * 4);
    L->rs_vals = (uint32_t*)dev_alloc(L, (size_t)max_mobile * 4);
    void* rs = dev_alloc(L, sort_scratch_bytes(max_mobile));
    if (!L->births || !L->rs_keys || !L->rs_vals || !rs) return PSC_E_NOMEM;
    sort_scratch_bind(L->rs_scratch, rs, max_mobile);

    if (L->opt.subvolume > 0) {
        auto& SV = L->subvol;
        const size_t nsub = (size_t)((L->ni + 1) / 2) * (size_t)((L->nj + 1) / 2) * (size_t)((L->nk + 1) / 2);
        SV.word = (uint32_t*)dev_alloc(L, nsub * 4);
        SV.head = (uint32_t*)dev_alloc(L, nsub * 4);
        SV.next = (uint32_t*)dev_alloc(L, (size_t)max_mobile * 4);
        SV.state = (uint32_t*)dev_alloc(L, (size_t)max_mobile * 4);
        SV.colour0 = (uint8_t*)dev_alloc(L, (size_t)max_mobile);
        SV.lead = (uint32_t*)dev_alloc(L, (size_t)max_mobile * 4);
        SV.lead_vox = (uint32_t*)dev_alloc(L, (size_t)max_mobile * 4);
        SV.counters = (uint32_t*)dev_alloc(L, 32 * 4);
        if (!SV.word || !SV.head || !SV.next || !SV.state || !SV.colour0 || !SV.lead || !SV.lead_vox ||
            !SV.counters)
            return PSC_E_NOMEM;
        SV.subvols = (int64_t)nsub;
        SV.slots = max_mobile;
        SV.blocks = subvol_max_blocks(L->sm_count);
        if (SV.blocks <= 0) return PSC_E_CUDA;
        launch_fill_u32(SV.word, kNoClaim, nsub, L->sm_count * 4, L->stream);
        launch_fill_u32(SV.head, kNoClaim, nsub, L->sm_count * 4, L->stream);
    }

    cudaStream_t st = L->stream;
    upload_stencil(st);
    int rc = cuda_fail(L, cudaMemcpyAsync(L->model_d, &M, sizeof(M), cudaMemcpyHostToDevice, st));
    if (rc) return rc;
    L->h2d += sizeof(M) + 5 * sizeof(uint32_t) + sizeof(Scalars);
    Scalars sh;
    std::memset(&sh, 0, sizeof(sh));
    for (int s = 0; s < L->nsp; ++s) sh.counts[s] = (int32_t)L->sp[s].n0;
    sh.next_id = (uint32_t)N;
    if ((rc = cuda_fail(L, cudaMemcpyAsync(L->sc, &sh, sizeof(sh), cudaMemcpyHostToDevice, st)))) return rc;
    if ((rc = cuda_fail(L, cudaMemsetAsync(L->occ, 0, V * sizeof(uint16_t), st)))) return rc;
    for (int x = 0; x < 2; ++x)
        if ((rc = cuda_fail(L, cudaMemsetAsync(L->dirty[x], 0, (size_t)L->dirty_words * 4, st)))) return rc;
    const int fill_blocks = L->sm_count * 8;
    uint8_t* labels_d = nullptr;
    if (comps) {
        // the labels are needed on the device only while placing
        labels_d = (uint8_t*)dev_alloc(L, V);
        if (!labels_d) return PSC_E_NOMEM;
        if ((rc = cuda_fail(L, cudaMemcpyAsync(labels_d, L->labels.data(), V, cudaMemcpyHostToDevice, st))))
            return rc;
        L->h2d += V;
        launch_mirror_walls(L->bits, nwords, nmirror, labels_d, L->geo, fill_blocks, st);
        L->launches += 1;
    } else if ((rc = cuda_fail(L, cudaMemsetAsync(L->bits, 0, nwords * sizeof(uint32_t), st)))) {
        return rc;
    }
    if (L->claim) launch_fill_u32(L->claim, kNoClaim, V, fill_blocks, st);
    for (int t = 0; t < 2; ++t)
        if (L->tables[t]) launch_fill_u64(L->tables[t], kEmptySlot, (size_t)1 << hb_max, fill_blocks, st);

    // ---- placement (Sec. 3.4): voxels in (Philox key, voxel) order, per
    // compartment, dealt to the species.  Only the first voxels of each
    // compartment matter: a histogram of the keys' top bits finds the bin
    // that covers them, and only the voxels up to it are sorted (by voxel,
    // then stably by key, then by compartment). ----
    if (N > 0) {
        const int nc = comps ? L->ncomp : 1;
        const int bins = 1 << kPlaceBits;
        int64_t need[kMaxCompartments] = {};
        for (int s = 0; s < L->nsp; ++s) need[comps ? L->sp[s].comp : 0] += L->sp[s].n0;
        uint32_t* hist = (uint32_t*)dev_alloc(L, (size_t)nc * bins * 4);
        int32_t* pick_n = (int32_t*)dev_alloc(L, 4);
        if (!hist || !pick_n) return PSC_E_NOMEM;
        if ((rc = cuda_fail(L, cudaMemsetAsync(hist, 0, (size_t)nc * bins * 4, st)))) return rc;
        if ((rc = cuda_fail(L, cudaMemsetAsync(pick_n, 0, 4, st)))) return rc;
        launch_place_hist((uint32_t)V, (uint32_t)seed, (uint32_t)(seed >> 32), labels_d, nc, hist, fill_blocks, st);
        std::vector<uint32_t> h((size_t)nc * bins);
        if ((rc = cuda_fail(L, cudaMemcpyAsync(h.data(), hist, h.size() * 4, cudaMemcpyDeviceToHost, st)))) return rc;
        if ((rc = cuda_fail(L, cudaStreamSynchronize(st)))) return rc;
        L->d2h += h.size() * 4;
        PlaceLimits lim;
        int64_t cand[kMaxCompartments] = {}, cbase[kMaxCompartments + 1] = {};
        for (int c = 0; c < kMaxCompartments; ++c) lim.bin[c] = -1;
        for (int c = 0; c < nc; ++c) {
            int64_t cum = 0;
            for (int b = 0; b < bins && need[c] > 0; ++b) {
                cum += h[(size_t)c * bins + b];
                if (cum >= need[c]) { lim.bin[c] = b; break; }
            }
            if (need[c] > 0 && lim.bin[c] < 0) return PSC_E_FULL;      // cannot happen: room was checked
            cand[c] = need[c] > 0 ? cum : 0;
            cbase[c + 1] = cbase[c] + cand[c];
        }
        const int64_t M = cbase[nc];
        {
            int64_t used[kMaxCompartments] = {};
            for (int s = 0; s < L->nsp; ++s) {
                const int c = comps ? L->sp[s].comp : 0;
                start[s] = cbase[c] + used[c];
                used[c] += L->sp[s].n0;
            }
        }
        uint32_t* cvox = (uint32_t*)dev_alloc(L, (size_t)M * 4);
        uint32_t* ckey = (uint32_t*)dev_alloc(L, (size_t)M * 4);
        void* scratch = dev_alloc(L, sort_scratch_bytes(M));
        if (!cvox || !ckey || !scratch) return PSC_E_NOMEM;
        SortScratch ss;
        sort_scratch_bind(ss, scratch, M);
        launch_place_pick((uint32_t)V, (uint32_t)seed, (uint32_t)(seed >> 32), labels_d, lim, cvox, ckey, pick_n,
                          (int32_t)M, &L->sc->err, fill_blocks, st);
        int vbits = 1;
        while (vbits < 31 && ((int64_t)1 << vbits) < L->V) ++vbits;
        if (radix_sort_pairs(cvox, ckey, nullptr, M, M, vbits, ss, st, &L->launches) != 0 ||
            radix_sort_pairs(ckey, cvox, nullptr, M, M, 32, ss, st, &L->launches) != 0)
            return cuda_fail(L, cudaErrorUnknown);
        if (comps) {
            launch_label_keys(cvox, labels_d, ckey, M, fill_blocks, st);
            if (radix_sort_pairs(ckey, cvox, nullptr, M, M, 8, ss, st, &L->launches) != 0)
                return cuda_fail(L, cudaErrorUnknown);
            L->launches += 1;
        }
        int64_t off[kMaxSpecies + 1];
        off[0] = 0;
        for (int s = 0; s < L->nsp; ++s) off[s + 1] = off[s] + L->sp[s].n0;
        launch_populate_scatter(cvox, N, off, start, L->nsp, L->occ, L->geo, L->model_d, fill_blocks, st);
        L->launches += 3;
        int32_t picked = 0;
        if ((rc = cuda_fail(L, cudaMemcpyAsync(&picked, pick_n, 4, cudaMemcpyDeviceToHost, st)))) return rc;
        if ((rc = cuda_fail(L, cudaStreamSynchronize(st)))) return rc;
        if (picked != M) return PSC_E_CUDA;                             // the two passes disagree
        dev_free_one(L, cvox);
        dev_free_one(L, ckey);
        dev_free_one(L, scratch);
        dev_free_one(L, hist);
        dev_free_one(L, pick_n);
    }
    if (labels_d) {
        if ((rc = cuda_fail(L, cudaStreamSynchronize(st)))) return rc;
        dev_free_one(L, labels_d);
    }
    if ((rc = cuda_fail(L, cudaStreamSynchronize(st)))) return rc;
    L->g = 0;
    L->clock = 0.0;
    L->populated = true;
    // the list-length estimates start from the placed counts (without the
    // pinned copy the grids follow the capacities)
    for (int s = 0; s < L->nsp; ++s) {
        L->est[s] = L->sp[s].n0;
        L->grid_class[s] = INT32_MAX;
    }
    L->counts_g = 0;
    if (!L->counts_h && cudaMallocHost(&L->counts_h, sizeof(int32_t) * kMaxSpecies) != cudaSuccess) {
        L->counts_h = nullptr;
        cudaGetLastError();
    }
    if (L->counts_h && !L->counts_ev &&
        cudaEventCreateWithFlags(&L->counts_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaFreeHost(L->counts_h);
        L->counts_h = nullptr;
        L->counts_ev = nullptr;
        cudaGetLastError();
    }
    // lists that start empty take the full grid until their first estimate
    if (L->counts_h)
        for (int s = 0; s < L->nsp; ++s)
            if (L->est[s] > 0) L->grid_class[s] = grid_class_for(L, s, L->est[s], 0);
    return L->clamped ? PSC_W_PCLAMP : PSC_OK;
}

}  // extern "C"

namespace psc_rt {

// The per-event grids a captured event takes (they follow the list estimates;
// so do the re-sort bounds, through the grid classes).
static void append_grids(const psc_lattice* L, std::vector<uint8_t>& key)
{
    for (int x = 0; x < L->nsp; ++x) {
        const int b = list_blocks(L, x);
        key.push_back((uint8_t)(b & 0xFF));
        key.push_back((uint8_t)(b >> 8));
    }
}

void graph_cache_clear(psc_lattice* L)
{
    for (auto& G : L->graphs)
        if (G.exec) cudaGraphExecDestroy(G.exec);
    L->graphs.clear();
    L->graph_seen.clear();
    for (auto& G : L->graphs1)
        if (G.exec) cudaGraphExecDestroy(G.exec);
    L->graphs1.clear();
    L->graph_seen1.clear();
}

// One event of species s (time t) replayed from a CUDA graph: its launches are
// fixed by the species, the event's parity, the claim tables' fill and whether
// the species' list is re-sorted after it; the event index comes from device
// memory.  Met for the first time, the event runs as usual; met again, it is
// captured once and replayed from then on.  For workloads whose runs of many
// events never recur (species with unrelated hop intervals), where launching
// dominates.  A failed capture turns graphs off for the lattice.
static int single_event(psc_lattice* L, int s, double t)
{
    auto finish = [&]() {
        L->sp[s].done++;
        L->g++;
        L->clock = t;
    };
    if (L->opt.graph_events < 2 || L->opt.time_kernels > 0 || L->g == UINT32_MAX - 1) {
        int rc = enqueue_event(L, s);
        finish();
        return rc;
    }
    // the re-sort counter runs out after this event (1: the list is re-sorted,
    // 2: its order does not pay, no re-sort)
    const uint8_t resort_now =
        (L->opt.resort_period > 0 && L->since_resort[s] + 1 >= (uint64_t)L->opt.resort_period)
            ? (sorted_order_pays(L, s) ? 1 : 2)
            : 0;
    std::vector<uint8_t> key;
    key.push_back((uint8_t)s);
    key.push_back((uint8_t)(L->g & 1u));
    key.push_back(resort_now);
    const uint8_t* tu = reinterpret_cast<const uint8_t*>(L->table_used);
    key.insert(key.end(), tu, tu + sizeof(L->table_used));
    append_grids(L, key);
    // the event index: events of species with reactions advance it on the
    // device, so a run of their replays sets it once
    auto set_index = [&]() {
        if (L->g_dev != (int64_t)L->g) {
            launch_fill_u32(&L->sc->g_base, L->g, 1, 1, L->stream);
            L->launches += 1;
        }
        L->g_dev = L->general[s] ? (int64_t)L->g + 1 : (int64_t)L->g;
    };
    for (const auto& G : L->graphs1) {
        if (G.key != key) continue;
        set_index();
        int rc = cuda_fail(L, cudaGraphLaunch(G.exec, L->stream));
        if (rc) return rc;
        L->table_used[0] = G.table_used[0];
        L->table_used[1] = G.table_used[1];
        L->since_resort[s] = resort_now ? 0 : L->since_resort[s] + 1;
        L->launches += G.launches;
        L->events += 1;
        finish();
        return PSC_OK;
    }
    if (std::find(L->graph_seen1.begin(), L->graph_seen1.end(), key) == L->graph_seen1.end()) {
        if (L->graph_seen1.size() >= 256) L->graph_seen1.erase(L->graph_seen1.begin());
        L->graph_seen1.push_back(key);
        int rc = enqueue_event(L, s);
        finish();
        return rc;
    }
    // seen before: capture once, then launch the graph
    const uint64_t since0 = L->since_resort[s];
    const uint32_t used0[2] = {L->table_used[0], L->table_used[1]};
    const int64_t launches0 = L->launches;
    const uint64_t events0 = L->events;
    const int sticky0 = L->sticky;
    auto restore = [&]() {
        L->since_resort[s] = since0;
        L->table_used[0] = used0[0];
        L->table_used[1] = used0[1];
        L->launches = launches0;
        L->events = events0;
        L->sticky = sticky0;
        L->opt.graph_events = 0;
        cudaGetLastError();
    };
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        L->capture_g0 = L->g;
        L->capture_single = true;
        int rc = enqueue_event(L, s);
        L->capture_g0 = -1;
        L->capture_single = false;
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(L->stream, &graph);
        if (rc == PSC_OK && ce == cudaSuccess && graph) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (rc != PSC_OK || ce != cudaSuccess) {
            if (exec) cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
    }
    if (!exec) {                                   // no graphs for this lattice: the ordinary way
        restore();
        int rc = enqueue_event(L, s);
        finish();
        return rc;
    }
    psc_lattice::GraphRun G;
    G.key = key;
    G.exec = exec;
    G.table_used[0] = L->table_used[0];
    G.table_used[1] = L->table_used[1];
    G.launches = L->launches - launches0;
    if (L->graphs1.size() >= 128) {
        cudaGraphExecDestroy(L->graphs1.front().exec);
        L->graphs1.erase(L->graphs1.begin());
    }
    L->graphs1.push_back(std::move(G));
    set_index();
    int rc = cuda_fail(L, cudaGraphLaunch(exec, L->stream));
    if (rc) return rc;
    finish();
    return PSC_OK;
}

// Runs of per-event launches replayed from CUDA graphs (psc_options.
// graph_events = K; small lattices, where launching dominates).  The next K
// events are planned with the scheduler; all must take per-event launches.
// Their pattern -- species in order, the claim tables' parity and fill, the
// re-sort counters -- fixes every launch but the event index, which the
// kernels then read from device memory.  A pattern met for the first time
// runs as usual; met again it is captured once and replayed from then on,
// the host bookkeeping advanced from what the capture recorded.  Any failure
// to capture turns graphs off for the lattice and leaves the events to the
// ordinary path.  *done = events queued (0: none, take one the ordinary way).
static int graph_run(psc_lattice* L, double t_end, int64_t room, int64_t* done)
{
    *done = 0;
    const int K = L->opt.graph_events;
    if (K < 2 || room < K || L->opt.time_kernels > 0 || (int64_t)L->g + K >= (int64_t)UINT32_MAX) return PSC_OK;
    uint64_t next[kMaxSpecies];
    for (int s = 0; s < L->nsp; ++s) next[s] = L->sp[s].done;
    std::vector<int> seq((size_t)K);
    std::vector<double> at((size_t)K);
    for (int e = 0; e < K; ++e) {
        int best = -1;
        double tb = 0.0;
        for (int s = 0; s < L->nsp; ++s) {
            if (!(L->sp[s].D > 0.0)) continue;
            const double t = (double)(next[s] + 1) * L->sp[s].tau;
            if (best < 0 || t < tb) { best = s; tb = t; }
        }
        if (best < 0 || tb > t_end) return PSC_OK;
        if (!L->general[best] && L->opt.persistent > 0) return PSC_OK;   // a stretch comes first
        seq[(size_t)e] = best;
        at[(size_t)e] = tb;
        next[best]++;
    }
    std::vector<uint8_t> key;
    auto put = [&key](const void* p, size_t n) {
        const uint8_t* b = static_cast<const uint8_t*>(p);
        key.insert(key.end(), b, b + n);
    };
    bool in_run[kMaxSpecies] = {};
    for (int s2 : seq) {
        key.push_back((uint8_t)s2);
        in_run[s2] = true;
    }
    const uint32_t parity = L->g & 1u;
    put(&parity, 4);
    put(L->table_used, sizeof(L->table_used));
    for (int s = 0; s < L->nsp; ++s)                 // only the run's species can re-sort in it
        if (in_run[s]) put(&L->since_resort[s], sizeof(uint64_t));
    append_grids(L, key);
    auto advance = [&](int e) {
        L->sp[seq[(size_t)e]].done++;
        L->g++;
        L->clock = at[(size_t)e];
    };
    for (const auto& G : L->graphs) {
        if (G.key != key) continue;
        launch_fill_u32(&L->sc->g_base, L->g, 1, 1, L->stream);
        L->g_dev = (int64_t)L->g;
        int rc = cuda_fail(L, cudaGraphLaunch(G.exec, L->stream));
        if (rc) return rc;
        for (int e = 0; e < K; ++e) advance(e);
        L->table_used[0] = G.table_used[0];
        L->table_used[1] = G.table_used[1];
        for (int s = 0; s < L->nsp; ++s)
            if (in_run[s]) L->since_resort[s] = G.since[(size_t)s];
        L->launches += G.launches + 1;
        L->events += (uint64_t)K;
        *done = K;
        return PSC_OK;
    }
    if (std::find(L->graph_seen.begin(), L->graph_seen.end(), key) == L->graph_seen.end()) {
        if (L->graph_seen.size() >= 32) L->graph_seen.erase(L->graph_seen.begin());
        L->graph_seen.push_back(key);
        for (int e = 0; e < K; ++e) {                // event by event, each from its own graph
            int rc = single_event(L, seq[(size_t)e], at[(size_t)e]);
            if (rc) return rc;
        }
        *done = K;
        return PSC_OK;
    }
    // seen before: capture once
    uint64_t done0[kMaxSpecies], since0[kMaxSpecies];
    for (int s = 0; s < L->nsp; ++s) { done0[s] = L->sp[s].done; since0[s] = L->since_resort[s]; }
    const uint32_t g0 = L->g, used0[2] = {L->table_used[0], L->table_used[1]};
    const double clock0 = L->clock;
    const int64_t launches0 = L->launches;
    const uint64_t events0 = L->events;
    const int sticky0 = L->sticky;
    auto restore = [&]() {
        for (int s = 0; s < L->nsp; ++s) { L->sp[s].done = done0[s]; L->since_resort[s] = since0[s]; }
        L->g = g0;
        L->table_used[0] = used0[0];
        L->table_used[1] = used0[1];
        L->clock = clock0;
        L->launches = launches0;
        L->events = events0;
        L->sticky = sticky0;
        L->opt.graph_events = 0;
        cudaGetLastError();
    };
    if (cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        restore();
        return PSC_OK;
    }
    L->capture_g0 = g0;
    int rc = PSC_OK;
    for (int e = 0; e < K && rc == PSC_OK; ++e) {
        rc = enqueue_event(L, seq[(size_t)e]);
        advance(e);
    }
    L->capture_g0 = -1;
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(L->stream, &graph);
    cudaGraphExec_t exec = nullptr;
    if (rc == PSC_OK && ce == cudaSuccess && graph) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != PSC_OK || ce != cudaSuccess || !exec) {
        if (exec) cudaGraphExecDestroy(exec);
        restore();
        return PSC_OK;
    }
    psc_lattice::GraphRun G;
    G.key = key;
    G.exec = exec;
    G.table_used[0] = L->table_used[0];
    G.table_used[1] = L->table_used[1];
    G.since.assign(L->since_resort, L->since_resort + L->nsp);
    G.launches = L->launches - launches0;
    if (L->graphs.size() >= 8) {
        cudaGraphExecDestroy(L->graphs.front().exec);
        L->graphs.erase(L->graphs.begin());
    }
    L->graphs.push_back(std::move(G));
    launch_fill_u32(&L->sc->g_base, g0, 1, 1, L->stream);
    L->g_dev = (int64_t)g0;
    if ((rc = cuda_fail(L, cudaGraphLaunch(exec, L->stream)))) return rc;
    L->launches += 1;
    *done = K;
    return PSC_OK;
}

// Queue events in scheduler order until max_events are queued or the next
// event lies after t_end.  Consecutive events of one species without
// reactions are grouped into persistent stretches (cut at re-sort points).
int drive(psc_lattice* L, double t_end, int64_t max_events)
{
    int64_t queued = 0;
    while (queued < max_events) {
        int s;
        double t;
        if (!next_event(L, &s, &t) || t > t_end) break;
        refresh_estimates(L);
        if (L->g == UINT32_MAX) return PSC_E_LIMIT;
        if (L->opt.subvolume > 0) {
            // the sub-volume rule: stretches of the species' events, one launch each
            const uint32_t g0 = L->g;
            const int64_t limit = std::max<int64_t>(
                1, std::min<int64_t>(std::min<int64_t>(max_events - queued, (int64_t)1 << 16),
                                     (int64_t)UINT32_MAX - L->g));
            int64_t e = 0;
            for (;;) {
                L->sp[s].done++;
                L->g++;
                L->clock = t;
                ++e;
                if (e >= limit) break;
                int s2;
                double t2;
                if (!next_event(L, &s2, &t2) || s2 != s || t2 > t_end) break;
                t = t2;
            }
            L->g = g0;
            int rc = enqueue_subvol(L, s, e);
            L->g = g0 + (uint32_t)e;
            if (rc) return rc;
            queued += e;
            continue;
        }
        int threads = 0, blocks = 0;
        const int per = run_width(L, s, &threads, &blocks);
        TilePlan plan{};
        // the tile kernel needs no molecule slots per thread: it also takes
        // species above the molecule-list kernel's capacity
        const bool tiles = L->opt.persistent > 0 && !L->general[s] && tile_plan(L, s, &plan);
        if (per > 0 || tiles) {
            // how long does species s stay next?  (Tile stretches keep their
            // own spatial order: no re-sort points.)
            const uint32_t g0 = L->g;
            int64_t limit = max_events - queued;
            if (L->opt.resort_period > 0 && !tiles)
                limit = std::min<int64_t>(limit, (int64_t)L->opt.resort_period - (int64_t)L->since_resort[s]);
            if (tiles) limit = std::min<int64_t>(limit, (int64_t)1 << 16);   // bounded launch length
            limit = std::max<int64_t>(1, std::min<int64_t>(limit, (int64_t)UINT32_MAX - L->g));
            int64_t e = 0;
            for (;;) {
                L->sp[s].done++;
                L->g++;
                L->clock = t;
                ++e;
                if (e >= limit) break;
                int s2;
                double t2;
                if (!next_event(L, &s2, &t2) || s2 != s || t2 > t_end) break;
                t = t2;
            }
            L->g = g0;                                   // event_args reads the first index
            int rc = tiles ? enqueue_tiles(L, s, e, plan) : enqueue_run(L, s, (int)e, per, threads, blocks);
            L->g = g0 + (uint32_t)e;
            if (rc) return rc;
            queued += e;
            if (tiles) continue;
            L->since_resort[s] += (uint64_t)e;
            if (L->opt.resort_period > 0 && L->since_resort[s] >= (uint64_t)L->opt.resort_period) {
                L->since_resort[s] = 0;
                if (sorted_order_pays(L, s)) {
                    cudaEvent_t sp = span_open(L);
                    rc = resort(L, s);
                    span_close(L, sp, kSpanResort);
                    if (rc) return rc;
                }
            }
            continue;
        }
        if (L->opt.graph_events > 1) {
            int64_t done = 0;
            int rc = graph_run(L, t_end, max_events - queued, &done);
            if (rc) return rc;
            if (done > 0) {
                queued += done;
                continue;
            }
        }
        int rc = single_event(L, s, t);
        if (rc) return rc;
        ++queued;
    }
    return PSC_OK;
}

}  // namespace psc_rt

extern "C" {

int psc_run(psc_lattice* L, double t_end)
{
    if (!L || !std::isfinite(t_end)) return PSC_E_ARG;
    if (!L->populated) return PSC_E_ORDER;
    if (L->sticky) return L->sticky;
    DevGuard dg(L->device);
    int rc = drive(L, t_end, INT64_MAX);
    if (rc) return rc;
    if (t_end > L->clock) L->clock = t_end;
    return PSC_OK;
}

int psc_run_events(psc_lattice* L, int64_t n_events)
{
    if (!L || n_events < 0) return PSC_E_ARG;
    if (!L->populated) return PSC_E_ORDER;
    if (L->sticky) return L->sticky;
    DevGuard dg(L->device);
    return drive(L, INFINITY, n_events);
}

int psc_synchronize(psc_lattice* L)
{
    if (!L) return PSC_E_ARG;
    DevGuard dg(L->device);
    return check_device(L);
}

int psc_counts(psc_lattice* L, int64_t* counts, int32_t n)
{
    if (!L || !counts || n < L->nsp) return PSC_E_ARG;
    for (int s = 0; s < n; ++s) counts[s] = s < L->nsp ? L->sp[s].n0 : 0;
    if (!L->populated) return PSC_OK;
    DevGuard dg(L->device);
    int rc = check_device(L);
    if (rc) return rc;
    int32_t c[kMaxSpecies];
    if ((rc = cuda_fail(L, cudaMemcpy(c, L->sc->counts, sizeof(c), cudaMemcpyDeviceToHost)))) return rc;
    L->d2h += sizeof(c);
    for (int s = 0; s < L->nsp; ++s) counts[s] = c[s];
    return PSC_OK;
}

static int read_list(psc_lattice* L, int32_t s, std::vector<int32_t>& vox, std::vector<uint32_t>& ids,
                     std::vector<uint64_t>* img)
{
    int rc = check_device(L);
    if (rc) return rc;
    int32_t n = 0;
    if ((rc = cuda_fail(L, cudaMemcpy(&n, &L->sc->counts[s], 4, cudaMemcpyDeviceToHost)))) return rc;
    L->d2h += 4 + (uint64_t)n * (img ? 16 : 8);
    const SpeciesList& l = L->model_h.lists[s];
    vox.resize(n);
    ids.resize(n);
    if (n > 0) {
        if ((rc = cuda_fail(L, cudaMemcpy(vox.data(), l.vox, (size_t)n * 4, cudaMemcpyDeviceToHost)))) return rc;
        if ((rc = cuda_fail(L, cudaMemcpy(ids.data(), l.ids, (size_t)n * 4, cudaMemcpyDeviceToHost)))) return rc;
        if (img) {
            img->resize(n);
            if ((rc = cuda_fail(L, cudaMemcpy(img->data(), l.img, (size_t)n * 8, cudaMemcpyDeviceToHost)))) return rc;
        }
    }
    return PSC_OK;
}

// The number of molecules of species s, for a call that only sizes its buffers
static int list_size(psc_lattice* L, int32_t s, int64_t* n_out)
{
    int rc = check_device(L);
    if (rc) return rc;
    int32_t n = 0;
    if ((rc = cuda_fail(L, cudaMemcpy(&n, &L->sc->counts[s], 4, cudaMemcpyDeviceToHost)))) return rc;
    L->d2h += 4;
    *n_out = n;
    return n > 0 ? PSC_E_ARG : PSC_OK;
}

// Read-out order by molecule id.  Ids are never reused, so when the ids of a
// list span exactly as many values as it has entries (every species without
// reactions keeps the ids placement gave it) each entry goes straight to
// its place; otherwise they are sorted.
static void order_by_id(const std::vector<uint32_t>& ids, std::vector<int64_t>& order)
{
    const int64_t n = (int64_t)ids.size();
    order.assign((size_t)n, -1);
    if (n == 0) return;
    const auto mm = std::minmax_element(ids.begin(), ids.end());
    const uint32_t lo = *mm.first;
    bool placed = (int64_t)*mm.second - (int64_t)lo + 1 == n;
    for (int64_t a = 0; placed && a < n; ++a) {
        int64_t& slot = order[ids[a] - lo];
        if (slot >= 0) placed = false;                   // a repeated id: sort instead
        slot = a;
    }
    if (placed) return;
    for (int64_t a = 0; a < n; ++a) order[a] = a;
    std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return ids[x] < ids[y]; });
}

// The n molecules of list s in id order, built on the device (ids sorted with
// their slots, then one gather) and copied to the caller's host buffers in
// one piece each.  Used when the list fits the re-sort scratch; returns
// PSC_OK, an error, or 1 when the caller should build the answer on the host.
static int device_positions(psc_lattice* L, int32_t s, int64_t n, bool unwrapped, int32_t* out,
                            uint32_t* ids_out)
{
    if (n <= 0 || n > L->rs_max) return 1;
    if (n > L->readout_cap) {
        if (L->readout) dev_free_one(L, L->readout);
        L->readout = (int32_t*)dev_alloc(L, (size_t)n * 16);
        L->readout_cap = L->readout ? n : 0;
        if (!L->readout) return 1;
    }
    int32_t* pos = L->readout;
    uint32_t* ids = reinterpret_cast<uint32_t*>(L->readout + 3 * n);
    const int blocks = event_blocks(L, n);
    if (readout_positions(L->model_h.lists[s], (int32_t)n, L->ni, L->nj, L->nk, unwrapped,
                          (L->bflags & PSC_FCC) != 0, L->rs_keys, L->rs_vals, L->rs_scratch, pos, ids, blocks,
                          L->stream, &L->launches) != 0)
        return cuda_fail(L, cudaErrorUnknown);
    int rc = cuda_fail(L, cudaMemcpyAsync(out, pos, (size_t)n * 12, cudaMemcpyDeviceToHost, L->stream));
    if (!rc && ids_out)
        rc = cuda_fail(L, cudaMemcpyAsync(ids_out, ids, (size_t)n * 4, cudaMemcpyDeviceToHost, L->stream));
    if (!rc) rc = cuda_fail(L, cudaStreamSynchronize(L->stream));
    if (rc) return rc;
    L->d2h += (uint64_t)n * (ids_out ? 16 : 12);
    return PSC_OK;
}

int psc_coords(psc_lattice* L, int32_t s, int32_t* ijk, uint32_t* ids_out, int64_t cap, int64_t* n_out)
{
    if (!L || !n_out || s < 0 || s >= L->nsp) return PSC_E_ARG;
    if (!L->populated) return PSC_E_ORDER;
    DevGuard dg(L->device);
    if (!ijk || cap <= 0) return list_size(L, s, n_out);
    int rc = list_size(L, s, n_out);               // E_ARG here only says the list is not empty
    if (rc != PSC_OK && rc != PSC_E_ARG) return rc;
    if (*n_out > cap) return PSC_E_ARG;
    if ((rc = device_positions(L, s, *n_out, false, ijk, ids_out)) <= 0) return rc;
    std::vector<int32_t> vox;
    std::vector<uint32_t> ids;
    rc = read_list(L, s, vox, ids, nullptr);
    if (rc) return rc;
    const int64_t n = (int64_t)vox.size();
    *n_out = n;
    if (n > cap) return PSC_E_ARG;
    std::vector<int64_t> order;
    order_by_id(ids, order);
    const uint32_t ni = (uint32_t)L->ni, nj = (uint32_t)L->nj;
    for (int64_t a = 0; a < n; ++a) {
        const uint32_t v = (uint32_t)vox[order[a]], q = v / ni;
        ijk[3 * a + 0] = (int32_t)(v - q * ni);
        ijk[3 * a + 1] = (int32_t)(q % nj);
        ijk[3 * a + 2] = (int32_t)(q / nj);
        if (ids_out) ids_out[a] = ids[order[a]];
    }
    return PSC_OK;
}

int psc_unwrapped(psc_lattice* L, int32_t s, int32_t* xyz, uint32_t* ids_out, int64_t cap, int64_t* n_out)
{
    if (!L || !n_out || s < 0 || s >= L->nsp) return PSC_E_ARG;
    if (!L->populated) return PSC_E_ORDER;
    DevGuard dg(L->device);
    if (!xyz || cap <= 0) return list_size(L, s, n_out);
    int rc = list_size(L, s, n_out);               // E_ARG here only says the list is not empty
    if (rc != PSC_OK && rc != PSC_E_ARG) return rc;
    if (*n_out > cap) return PSC_E_ARG;
    if ((rc = device_positions(L, s, *n_out, true, xyz, ids_out)) <= 0) return rc;
    std::vector<int32_t> vox;
    std::vector<uint32_t> ids;
    std::vector<uint64_t> img;
    rc = read_list(L, s, vox, ids, &img);
    if (rc) return rc;
    const int64_t n = (int64_t)vox.size();
    *n_out = n;
    if (n > cap) return PSC_E_ARG;
    std::vector<int64_t> order;
    order_by_id(ids, order);
    const uint32_t ni = (uint32_t)L->ni, nj = (uint32_t)L->nj;
    for (int64_t a = 0; a < n; ++a) {
        const uint32_t v = (uint32_t)vox[order[a]], q = v / ni;
        const uint64_t w = img[order[a]];
        const int32_t i = (int32_t)(v - q * ni), j = (int32_t)(q % nj), k = (int32_t)(q / nj);
        const int32_t I = i + (int32_t)(int16_t)(w & 0xFFFF) * L->ni;
        const int32_t J = j + (int32_t)(int16_t)((w >> 16) & 0xFFFF) * L->nj;
        const int32_t K = k + (int32_t)(int16_t)((w >> 32) & 0xFFFF) * L->nk;
        if (L->bflags & PSC_FCC) {
            const int32_t c3 = ((K % 3) + 3) % 3;
            xyz[3 * a + 0] = 2 * I + ((J + (c3 == 1 ? 1 : 0)) & 1);
            xyz[3 * a + 1] = 3 * J + c3;
        } else {
            xyz[3 * a + 0] = 2 * I + ((J + K) & 1);
            xyz[3 * a + 1] = 3 * J + (K & 1);
        }
        xyz[3 * a + 2] = K;
        if (ids_out) ids_out[a] = ids[order[a]];
    }
    return PSC_OK;
}

int psc_grid(psc_lattice* L, uint16_t* occ)
{
    if (!L || !occ) return PSC_E_ARG;
    if (!L->populated) return PSC_E_ORDER;
    DevGuard dg(L->device);
    int rc = check_device(L);
    if (rc) return rc;
    // exact codes: mirror-masked codes of species with reactions, then the
    // species without reactions from their lists
    uint16_t* tmp = (uint16_t*)dev_alloc(L, (size_t)L->V * 2);
    if (!tmp) return PSC_E_NOMEM;
    const int blocks = L->sm_count * 8;
    launch_materialize(tmp, L->occ, L->bits, L->mirror_n, L->labels.empty() ? 1 : L->ncomp, L->geo, L->V, blocks,
                       L->stream);
    for (int s = 0; s < L->nsp; ++s)
        if (!L->live[s])
            launch_scatter_codes(tmp, L->model_h.lists[s], &L->sc->counts[s], (uint16_t)(s + 1), blocks,
                                 L->stream);
    L->launches += 1;
    rc = cuda_fail(L, cudaStreamSynchronize(L->stream));
    if (!rc) rc = cuda_fail(L, cudaMemcpy(occ, tmp, (size_t)L->V * 2, cudaMemcpyDeviceToHost));
    L->d2h += (uint64_t)L->V * 2;
    dev_free_one(L, tmp);
    return rc;
}

int psc_time(const psc_lattice* L, double* t)
{
    if (!L || !t) return PSC_E_ARG;
    *t = L->clock;
    return PSC_OK;
}

int psc_event_index(const psc_lattice* L, uint32_t* g)
{
    if (!L || !g) return PSC_E_ARG;
    *g = L->g;
    return PSC_OK;
}

int psc_stats_get(psc_lattice* L, psc_stats* out)
{
    if (!L || !out) return PSC_E_ARG;
    std::memset(out, 0, sizeof(*out));
    out->events = L->events;
    out->launches = (uint64_t)L->launches;
    out->h2d_bytes = L->h2d;
    out->d2h_bytes = L->d2h;
    if (!L->populated) return PSC_OK;
    DevGuard dg(L->device);
    int rc = check_device(L);
    if (rc) return rc;
    unsigned long long st[kNumStats];
    if ((rc = cuda_fail(L, cudaMemcpy(st, L->sc->stats, sizeof(st), cudaMemcpyDeviceToHost)))) return rc;
    L->d2h += sizeof(st);
    out->attempts = st[kStatAttempts];
    out->hops = st[kStatHops];
    out->collisions = st[kStatCollisions];
    out->accepted = st[kStatAccepted];
    out->reactions2 = st[kStatReactions2];
    out->fires = st[kStatFires];
    out->reactions1 = st[kStatReactions1];
    out->births = st[kStatBirths];
    return PSC_OK;
}

int psc_set_options(psc_lattice* L, const psc_options* o)
{
    if (!L || !o) return PSC_E_ARG;
    if (o->block_threads && (o->block_threads < 32 || o->block_threads > 256 || (o->block_threads & 31)))
        return PSC_E_ARG;
    if (o->blocks_per_sm < 0) return PSC_E_ARG;
    graph_cache_clear(L);                            // captured launches follow the options
    if (o->resort_period) L->opt.resort_period = o->resort_period;
    if (o->block_threads) L->opt.block_threads = o->block_threads;
    if (o->blocks_per_sm) L->opt.blocks_per_sm = o->blocks_per_sm;
    if (o->collect_stats) L->opt.collect_stats = o->collect_stats;
    if (o->graph_events) L->opt.graph_events = o->graph_events < 0 ? 0 : o->graph_events;
    if (o->time_kernels) L->opt.time_kernels = o->time_kernels;
    if (o->claim_table) {
        if (o->claim_table < -1 || o->claim_table > 2) return PSC_E_ARG;
        if (L->populated) return PSC_E_ORDER;
        L->opt.claim_table = o->claim_table;
    }
    if (o->persistent) L->opt.persistent = o->persistent;
    if (o->run_per_thread) L->opt.run_per_thread = o->run_per_thread < 0 ? 0 : o->run_per_thread;
    if (o->barrier_timeout_us) {
        if (o->barrier_timeout_us < 0) return PSC_E_ARG;
        L->opt.barrier_timeout_us = o->barrier_timeout_us;
    }
    if (o->barrier_phantom) L->opt.barrier_phantom = o->barrier_phantom < 0 ? 0 : o->barrier_phantom;
    if (o->tiles) L->opt.tiles = o->tiles > 0 ? 1 : -1;
    if (o->subvolume) {
        if (L->populated) return PSC_E_ORDER;
        L->opt.subvolume = o->subvolume > 0 ? 1 : -1;
    }
    if (o->tile_regions) L->opt.tile_regions = o->tile_regions < 0 ? 0 : o->tile_regions;
    if (o->tile_lean) L->opt.tile_lean = o->tile_lean > 0 ? 1 : -1;
    if (o->slot_map) {
        if (o->slot_map < 1 || o->slot_map > 3) return PSC_E_ARG;
        L->opt.slot_map = o->slot_map;
    }
    if (o->claim_slots) {
        if (o->claim_slots < 2 || o->claim_slots > 64) return PSC_E_ARG;
        if (L->populated) return PSC_E_ORDER;
        L->opt.claim_slots = o->claim_slots;
    }
    return PSC_OK;
}

int psc_kernel_times_get(psc_lattice* L, psc_kernel_times* out)
{
    if (!L || !out) return PSC_E_ARG;
    std::memset(out, 0, sizeof(*out));
    DevGuard dg(L->device);
    cudaError_t e = cudaStreamSynchronize(L->stream);
    if (e != cudaSuccess) return cuda_fail(L, e);
    for (const auto& sp : L->spans) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, sp.a, sp.b) != cudaSuccess) ms = 0.0f;
        switch (sp.kind) {
        case kSpanClaim: out->claim_ms += ms; out->claim_launches++; break;
        case kSpanCommit: out->commit_ms += ms; out->commit_launches++; break;
        case kSpanReconcile: out->reconcile_ms += ms; out->reconcile_events++; break;
        case kSpanRun: out->run_ms += ms; out->run_launches++; out->run_events += sp.events; break;
        case kSpanTile:
        case kSpanTileLean:
            out->run_ms += ms; out->run_launches++; out->run_events += sp.events;
            out->tile_launches++; out->tile_events += sp.events;
            if (sp.kind == kSpanTileLean) out->tile_lean_events += sp.events;
            break;
        default: out->resort_ms += ms; out->resorts++; break;
        }
        L->event_pool.push_back(sp.a);
        L->event_pool.push_back(sp.b);
    }
    L->spans.clear();
    return PSC_OK;
}

int psc_device_bytes(const psc_lattice* L, int64_t* bytes)
{
    if (!L || !bytes) return PSC_E_ARG;
    const int64_t mirrors = L->labels.empty() ? 1 : L->ncomp;
    const int64_t mwords = (int64_t)mirror_words(L->ni, L->nj, L->nk);
    int64_t b = L->V * 2 + mwords * 4 * mirrors + 2 * ((mwords + 31) / 32) * 4 + (int64_t)sizeof(Scalars) +
                (int64_t)sizeof(ModelDev);
    if (L->claim) b += L->V * 4;
    b += 2 * L->table_slots * 8;
    int64_t N = 0;
    for (int s = 0; s < L->nsp; ++s) N += L->sp[s].n0;
    if (L->populated) {
        int64_t mx = 1, mm = 1;
        for (int s = 0; s < L->nsp; ++s) {
            b += (int64_t)L->cap[s] * 16;
            mx = std::max<int64_t>(mx, L->cap[s]);
            if (L->sp[s].D > 0.0) mm = std::max<int64_t>(mm, L->cap[s]);
        }
        b += mx * 24 + (int64_t)L->births_cap * (int64_t)sizeof(Birth) + mm * 8 +
             (int64_t)sort_scratch_bytes(mm);
    } else {
        b += 2 * N * 16 + 2 * N * 8;
    }
    // sub-volume rule buffers
    b += L->subvol.subvols * 8 + L->subvol.slots * 17 + (L->subvol.counters ? 128 : 0);
    // tile kernel buffers, once a stretch has used them
    const auto& T = L->tile;
    b += T.slots * 4 * 5 + (int64_t)T.regions * 4 * 4 + T.ids * 8 + T.halo_entries * (int64_t)sizeof(uint2);
    if (T.claim) b += L->V * 4;
    b += L->readout_cap * 16;                        // staging of the device-side read-out, once used
    *bytes = b;
    return PSC_OK;
}

void psc_lattice_destroy(psc_lattice* L)
{
    if (!L) return;
    {
        DevGuard dg(L->device);
        if (L->stream) cudaStreamSynchronize(L->stream);
        for (const auto& sp : L->spans) { cudaEventDestroy(sp.a); cudaEventDestroy(sp.b); }
        for (cudaEvent_t ev : L->event_pool) cudaEventDestroy(ev);
        if (L->counts_ev) cudaEventDestroy(L->counts_ev);
        if (L->counts_h) cudaFreeHost(L->counts_h);
        graph_cache_clear(L);
        dev_free_all(L);
        if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
    }
    delete L;
}

}  // extern "C"
