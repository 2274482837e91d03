// psc_batch.cpp -- batches of lattices advanced by shared launches, and the
// serving loop built on them (continuous batching with admission by device
// memory).  Each member of a batch keeps its own scheduler (Sec. 2.2); one
// batched launch per event phase covers every member's next event.
#include "psc.h"
#include "psc_internal.h"
#include "psc_runtime.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

using namespace psc;
using namespace psc_rt;

namespace {

constexpr int kItemBlocksMaxDefault = 64;   // blocks per member per launch (grid-stride inside)
constexpr int kItemThreadsDefault = 256;   // threads per block of the batched launches

struct Member {
    psc_lattice* L = nullptr;
    double t_stop = INFINITY;             // run events up to this time
};

}  // namespace

struct psc_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Member slot[kBatchMax];
    int32_t size = 0;
    EventArgs* tmpl_ev = nullptr;         // [kBatchMax][kMaxSpecies] on the device
    ReconcileArgs* tmpl_rc = nullptr;
    int64_t launches = 0;
    int threads = kItemThreadsDefault;
    int item_blocks_max = kItemBlocksMaxDefault;
    int32_t resort_period = -1;           // events of a member's species between Morton re-sorts (-1 never)
};

namespace {

int item_blocks(const psc_batch* B, int64_t work)
{
    const int64_t b = (work + B->threads - 1) / B->threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, B->item_blocks_max));
}

// Queue the next event of every member whose next event time is <= its
// t_stop (and <= t_cap); returns how many members had one.
int batch_event(psc_batch* B, double t_cap, int* rc_out)
{
    *rc_out = PSC_OK;
    struct Act {
        int slot, s;
        double t;
    };
    Act acts[kBatchMax];
    int na = 0;
    static thread_local BatchLaunch bl;
    bl.n = 0;
    int total = 0;
    for (int i = 0; i < kBatchMax; ++i) {
        psc_lattice* L = B->slot[i].L;
        if (!L || L->sticky) continue;
        int s;
        double t;
        if (!next_event(L, &s, &t) || t > B->slot[i].t_stop || t > t_cap || L->g == UINT32_MAX) continue;
        acts[na++] = {i, s, t};
        BatchItem& it = bl.item[bl.n++];
        it.rep = i;
        it.sel = s;
        it.g = L->g;
        it.block0 = total;
        it.mask = 0;
        total += item_blocks(B, L->cap[s]);
    }
    if (na == 0) return 0;
    bl.total_blocks = total;
    launch_claim_batch(B->tmpl_ev, bl, B->threads, B->stream);
    launch_commit_batch(B->tmpl_ev, bl, B->threads, B->stream);
    B->launches += 2;
    // list passes: the k-th partner list of each member's event checked
    // against the member's grid (list 0 is the member's own species, whose
    // commit noted its leavers), then every list of every member's event
    // filled, a block each; a list's scratch range follows those of the lists
    // before it in the member's order
    for (int k = 1;; ++k) {
        bl.n = 0;
        total = 0;
        for (int a = 0; a < na; ++a) {
            psc_lattice* L = B->slot[acts[a].slot].L;
            const std::vector<int>& rec = L->reconcile[acts[a].s];
            if (k >= (int)rec.size()) continue;
            BatchItem& it = bl.item[bl.n++];
            it.rep = acts[a].slot;
            it.sel = rec[k];
            it.g = L->g;                  // the event's parity picks the commit's dirty map
            it.block0 = total;
            it.mask = 0;
            for (int q = 0; q < k; ++q) it.mask |= 1u << rec[q];
            total += item_blocks(B, L->cap[rec[k]]);
        }
        if (bl.n == 0) break;
        bl.total_blocks = total;
        launch_reconcile_batch(B->tmpl_rc, bl, B->threads, B->stream);
        B->launches += 1;
    }
    bl.n = 0;
    for (int a = 0; a < na; ++a) {
        psc_lattice* L = B->slot[acts[a].slot].L;
        const std::vector<int>& rec = L->reconcile[acts[a].s];
        uint32_t before = 0;
        for (int x : rec) {
            BatchItem& it = bl.item[bl.n++];
            it.rep = acts[a].slot;
            it.sel = x;
            it.g = L->g;
            it.block0 = bl.n - 1;
            it.mask = before;
            before |= 1u << x;
            if (bl.n == kBatchMax) {
                bl.total_blocks = bl.n;
                launch_fill_batch(B->tmpl_rc, bl, B->stream);
                B->launches += 1;
                bl.n = 0;
            }
        }
    }
    if (bl.n > 0) {
        bl.total_blocks = bl.n;
        launch_fill_batch(B->tmpl_rc, bl, B->stream);
        B->launches += 1;
    }
    bl.n = 0;
    for (int a = 0; a < na; ++a) {
        psc_lattice* L = B->slot[acts[a].slot].L;
        if (!L->fo2[acts[a].s]) continue;
        BatchItem& it = bl.item[bl.n];
        it.rep = acts[a].slot;
        it.sel = acts[a].s;
        it.g = L->g;
        it.block0 = bl.n;
        it.mask = 0;
        bl.n++;
    }
    if (bl.n > 0) {
        bl.total_blocks = bl.n;
        launch_births_batch(B->tmpl_ev, bl, B->stream);
        B->launches += 1;
    }
    const cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        *rc_out = PSC_E_CUDA;
        return na;
    }
    for (int a = 0; a < na; ++a) {
        psc_lattice* L = B->slot[acts[a].slot].L;
        L->sp[acts[a].s].done++;
        L->g++;
        L->clock = acts[a].t;
        L->events++;
        L->launches += 2;
        // the member's list in Morton order again every resort_period of its events (the order of a
        // list never changes results)
        if (B->resort_period > 0 && ++L->since_resort[acts[a].s] >= (uint64_t)B->resort_period) {
            L->since_resort[acts[a].s] = 0;
            const int rc = psc_rt::resort(L, acts[a].s);
            if (rc) {
                *rc_out = rc;
                return na;
            }
        }
    }
    return na;
}

int upload_templates(psc_batch* B, int slot, psc_lattice* L)
{
    std::vector<EventArgs> ev(kMaxSpecies);
    std::vector<ReconcileArgs> rc(kMaxSpecies);
    for (int s = 0; s < L->nsp; ++s) {
        ev[s] = event_args(L, s);
        rc[s] = reconcile_args(L, s);
    }
    if (cudaMemcpy(B->tmpl_ev + (size_t)slot * kMaxSpecies, ev.data(), sizeof(EventArgs) * kMaxSpecies,
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return PSC_E_CUDA;
    if (cudaMemcpy(B->tmpl_rc + (size_t)slot * kMaxSpecies, rc.data(), sizeof(ReconcileArgs) * kMaxSpecies,
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return PSC_E_CUDA;
    L->h2d += sizeof(EventArgs) * kMaxSpecies + sizeof(ReconcileArgs) * kMaxSpecies;
    return PSC_OK;
}

int batch_add_until(psc_batch* B, psc_lattice* L, double t_stop)
{
    if (!B || !L) return PSC_E_ARG;
    if (!L->populated) return PSC_E_ORDER;
    if (L->device != B->device || L->stream != B->stream || !L->claim || L->tables[0]) return PSC_E_UNSUPPORTED;
    int free_slot = -1;
    for (int i = 0; i < kBatchMax; ++i) {
        if (B->slot[i].L == L) return PSC_E_ARG;
        if (!B->slot[i].L && free_slot < 0) free_slot = i;
    }
    if (free_slot < 0) return PSC_E_CAPACITY;
    DevGuard dg(B->device);
    int rc = upload_templates(B, free_slot, L);
    if (rc) return rc;
    B->slot[free_slot].L = L;
    B->slot[free_slot].t_stop = t_stop;
    B->size++;
    return PSC_OK;
}

}  // namespace

extern "C" {

int psc_batch_create(psc_batch** out, int device, void* cuda_stream)
{
    if (!out || device < 0) return PSC_E_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) return PSC_E_CUDA;
    psc_batch* B = new (std::nothrow) psc_batch();
    if (!B) return PSC_E_NOMEM;
    B->device = device;
    DevGuard dg(device);
    if (cuda_stream) {
        B->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) { delete B; return PSC_E_CUDA; }
        B->own_stream = true;
    }
    if (cudaMalloc(&B->tmpl_ev, sizeof(EventArgs) * kBatchMax * kMaxSpecies) != cudaSuccess ||
        cudaMalloc(&B->tmpl_rc, sizeof(ReconcileArgs) * kBatchMax * kMaxSpecies) != cudaSuccess) {
        cudaFree(B->tmpl_ev);
        if (B->own_stream) cudaStreamDestroy(B->stream);
        delete B;
        return PSC_E_NOMEM;
    }
    *out = B;
    return PSC_OK;
}

int psc_batch_add(psc_batch* B, psc_lattice* L) { return batch_add_until(B, L, INFINITY); }

int psc_batch_remove(psc_batch* B, psc_lattice* L)
{
    if (!B || !L) return PSC_E_ARG;
    for (int i = 0; i < kBatchMax; ++i) {
        if (B->slot[i].L == L) {
            B->slot[i].L = nullptr;
            B->size--;
            return PSC_OK;
        }
    }
    return PSC_E_ARG;
}

int psc_batch_size(const psc_batch* B, int32_t* n)
{
    if (!B || !n) return PSC_E_ARG;
    *n = B->size;
    return PSC_OK;
}

int64_t psc_batch_launches(const psc_batch* B) { return B ? B->launches : 0; }

int psc_batch_run_events(psc_batch* B, int64_t n_events)
{
    if (!B || n_events < 0) return PSC_E_ARG;
    DevGuard dg(B->device);
    // every member with events left takes part in each batched event
    for (int64_t e = 0; e < n_events; ++e) {
        int rc;
        if (batch_event(B, INFINITY, &rc) == 0) break;
        if (rc) return rc;
    }
    return PSC_OK;
}

int psc_batch_run(psc_batch* B, double t_end)
{
    if (!B || !std::isfinite(t_end)) return PSC_E_ARG;
    DevGuard dg(B->device);
    for (;;) {
        int rc;
        if (batch_event(B, t_end, &rc) == 0) break;
        if (rc) return rc;
    }
    for (int i = 0; i < kBatchMax; ++i) {
        psc_lattice* L = B->slot[i].L;
        if (L && t_end > L->clock) L->clock = t_end;
    }
    return PSC_OK;
}

// Block shape of the batched launches, tuned by timing batched events.  Like
// the lattice tuner it changes only how work is laid out on the GPU, so the
// trial rounds are real events of every member.
int psc_batch_autotune(psc_batch* B, int64_t max_rounds, psc_batch_tune_result* out)
{
    if (!B || !out || max_rounds < 0) return PSC_E_ARG;
    std::memset(out, 0, sizeof(*out));
    DevGuard dg(B->device);
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return PSC_E_CUDA;
    }
    const int64_t W = std::max<int64_t>(2, std::min<int64_t>(64, max_rounds / 14));
    int64_t budget = max_rounds;
    int rc = PSC_OK;
    // run up to n batched events; *us = microseconds per batched event (timed)
    auto rounds = [&](int64_t n, bool time_it, double* us) -> int {
        n = std::min(n, budget);
        int64_t done = 0;
        if (time_it && cudaEventRecord(a, B->stream) != cudaSuccess) return PSC_E_CUDA;
        for (; done < n; ++done) {
            int r;
            if (batch_event(B, INFINITY, &r) == 0) break;
            if (r) return r;
        }
        budget -= done;
        out->rounds += done;
        if (!time_it) return PSC_OK;
        if (cudaEventRecord(b, B->stream) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess)
            return PSC_E_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) return PSC_E_CUDA;
        out->trials++;
        *us = done > 0 ? 1e3 * (double)ms / (double)done : INFINITY;
        return PSC_OK;
    };
    int best_t = B->threads, best_m = B->item_blocks_max;
    double best_us = INFINITY;
    rc = rounds(1, false, nullptr);
    if (!rc) rc = rounds(W, true, &best_us);
    out->us_per_round_before = best_us;
    const int threads[] = {128, 256};
    const int per_member[] = {8, 16, 32, 64, 128, 256};
    for (int th : threads) {
        for (int m : per_member) {
            if (rc || budget <= 0) break;
            if (th == best_t && m == best_m) continue;
            B->threads = th;
            B->item_blocks_max = m;
            double us;
            if (!(rc = rounds(W, true, &us)) && us < best_us) { best_us = us; best_t = th; best_m = m; }
        }
    }
    B->threads = best_t;
    B->item_blocks_max = best_m;
    // the members' re-sort period: none, or every 64 or 256 of a member's
    // events; each trial spans at least one period of the fastest member
    int best_r = B->resort_period;
    for (const int period : {-1, 64, 256}) {
        if (rc || budget <= 0) break;
        if (period == best_r) continue;
        B->resort_period = period;
        double us;
        const int64_t span = period > 0 ? std::max<int64_t>(W, period) : W;
        if (!(rc = rounds(span, true, &us)) && us < best_us) { best_us = us; best_r = period; }
    }
    B->resort_period = best_r;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    out->threads = best_t;
    out->blocks_per_member = best_m;
    out->resort_period = best_r;
    out->us_per_round = best_us;
    return rc;
}

void psc_batch_destroy(psc_batch* B)
{
    if (!B) return;
    {
        DevGuard dg(B->device);
        cudaStreamSynchronize(B->stream);
        cudaFree(B->tmpl_ev);
        cudaFree(B->tmpl_rc);
        if (B->own_stream) cudaStreamDestroy(B->stream);
    }
    delete B;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// serving loop
// ---------------------------------------------------------------------------
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket = 0;
    psc_request r{};
    std::vector<double> D, k;
    std::vector<int64_t> n0;
    std::vector<int32_t> nre, re, npr, pr;
    Clock::time_point submitted;
};

struct Running {
    psc_lattice* L = nullptr;
    int64_t ticket = 0;
    int64_t bytes = 0;
    double t_end = 0.0;
    int32_t n_species = 0;
    Clock::time_point submitted;
};

struct Outcome {
    int status = PSC_OK;
    std::vector<int64_t> counts;
    double seconds = 0.0;
};

// create and populate a lattice for a request; *bytes = its device footprint
int build_lattice(const Request& q, int device, cudaStream_t stream, psc_lattice** out)
{
    const psc_request& r = q.r;
    psc_lattice* L = nullptr;
    int rc = psc_lattice_create(&L, r.ni, r.nj, r.nk, r.voxel_radius_m, r.boundary_flags, device, stream);
    if (rc) return rc;
    psc_options o{};
    o.claim_table = 1;
    o.resort_period = -1;
    psc_set_options(L, &o);
    for (int s = 0; s < r.n_species && !rc; ++s) rc = psc_add_species(L, q.D[s], q.n0[s], nullptr);
    for (int x = 0; x < r.n_reactions && !rc; ++x)
        rc = psc_add_reaction(L, &q.re[2 * x], q.nre[x], &q.pr[2 * x], q.npr[x], q.k[x], nullptr);
    if (rc) {
        psc_lattice_destroy(L);
        return rc;
    }
    *out = L;
    return PSC_OK;
}

}  // namespace

struct psc_server {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t max_bytes = 0;
    int64_t used = 0;
    int64_t peak = 0;
    int32_t max_active = 0;
    psc_batch* batch = nullptr;
    int64_t next_ticket = 1;
    std::deque<Request> queue;
    std::vector<Running> running;
    std::map<int64_t, Outcome> done;
};

extern "C" {

int psc_server_create(psc_server** out, int device, void* cuda_stream, int64_t max_device_bytes, int32_t max_active)
{
    if (!out || max_device_bytes <= 0 || max_active < 1) return PSC_E_ARG;
    *out = nullptr;
    psc_server* S = new (std::nothrow) psc_server();
    if (!S) return PSC_E_NOMEM;
    S->device = device;
    S->max_bytes = max_device_bytes;
    S->max_active = std::min<int32_t>(max_active, kBatchMax);
    {
        DevGuard dg(device);
        if (cuda_stream) {
            S->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
                delete S;
                return PSC_E_CUDA;
            }
            S->own_stream = true;
        }
    }
    int rc = psc_batch_create(&S->batch, device, S->stream);
    if (rc) {
        if (S->own_stream) cudaStreamDestroy(S->stream);
        delete S;
        return rc;
    }
    *out = S;
    return PSC_OK;
}

int psc_server_submit(psc_server* S, const psc_request* r, int64_t* ticket)
{
    if (!S || !r || !ticket) return PSC_E_ARG;
    if (r->n_species < 1 || r->n_species > kMaxSpecies || r->n_reactions < 0 || r->n_reactions > kMaxReactions ||
        !r->D || !r->initial_count || !std::isfinite(r->t_end))
        return PSC_E_ARG;
    if (r->n_reactions > 0 && (!r->n_reactants || !r->reactants || !r->n_products || !r->k)) return PSC_E_ARG;
    Request q;
    q.r = *r;
    q.D.assign(r->D, r->D + r->n_species);
    q.n0.assign(r->initial_count, r->initial_count + r->n_species);
    q.nre.assign(r->n_reactions, 0);
    q.npr.assign(r->n_reactions, 0);
    q.re.assign(2 * (size_t)r->n_reactions, 0);
    q.pr.assign(2 * (size_t)r->n_reactions, 0);
    q.k.assign(r->n_reactions, 0.0);
    for (int x = 0; x < r->n_reactions; ++x) {
        q.nre[x] = r->n_reactants[x];
        q.npr[x] = r->n_products[x];
        if (q.nre[x] < 1 || q.nre[x] > 2 || q.npr[x] < 0 || q.npr[x] > 2) return PSC_E_ARG;
        for (int a = 0; a < q.nre[x]; ++a) q.re[2 * x + a] = r->reactants[2 * x + a];
        for (int a = 0; a < q.npr[x]; ++a) q.pr[2 * x + a] = r->products[2 * x + a];
        q.k[x] = r->k[x];
    }
    q.ticket = S->next_ticket++;
    q.submitted = Clock::now();
    *ticket = q.ticket;
    S->queue.push_back(std::move(q));
    return PSC_OK;
}

int psc_server_step(psc_server* S, int32_t n_events, int32_t* n_active, int32_t* n_waiting)
{
    if (!S || n_events < 0) return PSC_E_ARG;
    DevGuard dg(S->device);
    // admit in arrival order while memory and slots allow
    while (!S->queue.empty() && (int32_t)S->running.size() < S->max_active) {
        Request& q = S->queue.front();
        psc_lattice* L = nullptr;
        int rc = build_lattice(q, S->device, S->stream, &L);
        if (rc) {
            Outcome& o = S->done[q.ticket];
            o.status = rc;
            S->queue.pop_front();
            continue;
        }
        int64_t bytes = 0;
        psc_device_bytes(L, &bytes);
        if (S->used + bytes > S->max_bytes) {
            psc_lattice_destroy(L);
            if (S->running.empty()) {          // can never fit
                Outcome& o = S->done[q.ticket];
                o.status = PSC_E_NOMEM;
                S->queue.pop_front();
                continue;
            }
            break;
        }
        rc = psc_populate(L, q.r.seed);
        if (rc < 0) {
            psc_lattice_destroy(L);
            Outcome& o = S->done[q.ticket];
            o.status = rc;
            S->queue.pop_front();
            continue;
        }
        psc_device_bytes(L, &bytes);
        rc = batch_add_until(S->batch, L, q.r.t_end);
        if (rc) {
            psc_lattice_destroy(L);
            Outcome& o = S->done[q.ticket];
            o.status = rc;
            S->queue.pop_front();
            continue;
        }
        Running run;
        run.L = L;
        run.ticket = q.ticket;
        run.bytes = bytes;
        run.t_end = q.r.t_end;
        run.n_species = q.r.n_species;
        run.submitted = q.submitted;
        S->running.push_back(run);
        S->used += bytes;
        S->peak = std::max(S->peak, S->used);
        S->queue.pop_front();
    }
    // advance every running simulation by up to n_events of its events
    for (int32_t e = 0; e < n_events; ++e) {
        int rc;
        if (batch_event(S->batch, INFINITY, &rc) == 0) break;
        if (rc) return rc;
    }
    // retire the finished ones
    for (size_t x = 0; x < S->running.size();) {
        Running& run = S->running[x];
        int s;
        double t;
        const bool more = next_event(run.L, &s, &t) && t <= run.t_end && run.L->g != UINT32_MAX;
        if (more && !run.L->sticky) {
            ++x;
            continue;
        }
        Outcome& o = S->done[run.ticket];
        o.counts.assign(run.n_species, 0);
        o.status = run.L->sticky ? run.L->sticky : psc_counts(run.L, o.counts.data(), run.n_species);
        o.seconds = std::chrono::duration<double>(Clock::now() - run.submitted).count();
        psc_batch_remove(S->batch, run.L);
        psc_lattice_destroy(run.L);
        S->used -= run.bytes;
        run = S->running.back();
        S->running.pop_back();
    }
    if (n_active) *n_active = (int32_t)S->running.size();
    if (n_waiting) *n_waiting = (int32_t)S->queue.size();
    return PSC_OK;
}

int psc_server_result(psc_server* S, int64_t ticket, int64_t* counts, int32_t n, double* seconds)
{
    if (!S) return PSC_E_ARG;
    auto it = S->done.find(ticket);
    if (it == S->done.end()) return PSC_E_ORDER;
    const Outcome& o = it->second;
    if (o.status < 0) return o.status;
    if (counts) {
        if (n < (int32_t)o.counts.size()) return PSC_E_ARG;
        for (size_t s = 0; s < o.counts.size(); ++s) counts[s] = o.counts[s];
    }
    if (seconds) *seconds = o.seconds;
    return PSC_OK;
}

int psc_server_memory(const psc_server* S, int64_t* in_use, int64_t* peak)
{
    if (!S) return PSC_E_ARG;
    if (in_use) *in_use = S->used;
    if (peak) *peak = S->peak;
    return PSC_OK;
}

void psc_server_destroy(psc_server* S)
{
    if (!S) return;
    {
        DevGuard dg(S->device);
        cudaStreamSynchronize(S->stream);
        for (Running& run : S->running) psc_lattice_destroy(run.L);
        psc_batch_destroy(S->batch);
        if (S->own_stream) cudaStreamDestroy(S->stream);
    }
    delete S;
}

}  // extern "C"
