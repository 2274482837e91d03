// psc_slab.cpp -- slabs of a lattice along k with ghost layers and per-event
// exchanges (the paper's sub-domains with ghost voxels, Sec. 2.5), for
// stretches of events of one species without reactions: the C ABI of
// include/psc.h (psc_slab_*), the kernels are in psc_slab.cuh.
#include "psc.h"
#include "psc_runtime.h"

#include <cstring>
#include <new>
#include <vector>

using namespace psc;
using namespace psc_rt;

struct psc_slab {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    int32_t index = 0, count = 1;
    int32_t species = 0;
    uint64_t seed = 0;
    uint32_t g = 0;                    // next event index
    SlabArgs a{};
    size_t claim_bytes = 0, commit_bytes = 0;
    // exchange buffers owned by the slab ([0] lower side, [1] upper side)
    void* own[8] = {};
    psc_slab_buffers buf{};
    std::vector<void*> allocs;
    int sticky = PSC_OK;
};

namespace {

void* slab_alloc(psc_slab* S, size_t bytes)
{
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) return nullptr;
    S->allocs.push_back(p);
    return p;
}

int slab_fail(psc_slab* S, cudaError_t e)
{
    if (e == cudaSuccess) return PSC_OK;
    if (!S->sticky) S->sticky = PSC_E_CUDA;
    return PSC_E_CUDA;
}

int slab_blocks(const psc_slab* S, int64_t work)
{
    int64_t b = (work + 255) / 256;
    const int64_t most = (int64_t)S->sm_count * 8;
    return (int)(b < 1 ? 1 : (b > most ? most : b));
}

// point the kernels' message pointers at the current buffers
void bind(psc_slab* S)
{
    for (int side = 0; side < 2; ++side) {
        S->a.send_commit[side] = static_cast<uint8_t*>(S->buf.send_commit[side]);
        S->a.recv_commit[side] = static_cast<const uint8_t*>(S->buf.recv_commit[side]);
        S->a.recv_claim[side] = static_cast<const uint32_t*>(S->buf.recv_claim[side]);
    }
}

int check(psc_slab* S)
{
    if (S->sticky) return S->sticky;
    int32_t err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, S->a.err, 4, cudaMemcpyDeviceToHost, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess) return slab_fail(S, e);
    if (err) S->sticky = PSC_E_CAPACITY;
    return S->sticky;
}

}  // namespace

extern "C" int psc_slab_create(psc_slab** out, psc_lattice* L, int32_t species, int32_t index, int32_t count,
                               int device, void* cuda_stream)
{
    if (!out || !L || count < 1 || index < 0 || index >= count) return PSC_E_ARG;
    *out = nullptr;
    if (!L->populated) return PSC_E_ORDER;
    if (species < 0 || species >= L->nsp) return PSC_E_ARG;
    if (L->bflags & PSC_FCC) return PSC_E_UNSUPPORTED;
    // one mobile species without reactions; every other species immobile
    if (!(L->sp[species].D > 0.0) || L->general[species] || L->live[species]) return PSC_E_UNSUPPORTED;
    for (int s = 0; s < L->nsp; ++s)
        if (s != species && L->sp[s].D > 0.0) return PSC_E_UNSUPPORTED;
    if (L->nk % count) return PSC_E_DIMS;
    const int32_t m = L->nk / count;
    if (m < 2) return PSC_E_DIMS;

    // the lattice's state on the host
    int rc = psc_synchronize(L);
    if (rc) return rc;
    std::vector<uint16_t> occ((size_t)L->V);
    if ((rc = psc_grid(L, occ.data()))) return rc;
    int64_t n = 0;
    rc = psc_unwrapped(L, species, nullptr, nullptr, 0, &n);     // sizing: E_ARG when n > 0
    if (rc != PSC_OK && rc != PSC_E_ARG) return rc;
    std::vector<int32_t> ijk((size_t)std::max<int64_t>(1, n) * 3), xyz((size_t)std::max<int64_t>(1, n) * 3);
    std::vector<uint32_t> ids((size_t)std::max<int64_t>(1, n));
    if (n > 0) {
        if ((rc = psc_coords(L, species, ijk.data(), ids.data(), n, &n))) return rc;
        if ((rc = psc_unwrapped(L, species, xyz.data(), nullptr, n, &n))) return rc;
    }
    uint32_t g0 = 0;
    psc_event_index(L, &g0);

    psc_slab* S = new (std::nothrow) psc_slab();
    if (!S) return PSC_E_NOMEM;
    S->device = device;
    S->index = index;
    S->count = count;
    S->species = species;
    S->seed = L->seed;
    S->g = g0;
    DevGuard dg(device);
    if (cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete S;
        return PSC_E_CUDA;
    }
    if (cuda_stream) {
        S->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete S;
            return PSC_E_CUDA;
        }
        S->own_stream = true;
    }
    upload_stencil(S->stream);

    SlabArgs& a = S->a;
    a.ni = L->ni; a.nj = L->nj; a.nk = L->nk; a.m = m; a.k0 = index * m;
    a.bflags = L->bflags & PSC_PERIODIC_ALL;
    const uint32_t nij = (uint32_t)L->ni * (uint32_t)L->nj;
    a.lw = (nij + 31) / 32;
    const bool kper = (a.bflags & PSC_PERIODIC_K) != 0;
    a.has[0] = (kper || index > 0) ? 1 : 0;
    a.has[1] = (kper || index < count - 1) ? 1 : 0;
    a.key0 = (uint32_t)L->seed;
    a.key1 = (uint32_t)(L->seed >> 32);
    a.s = (uint32_t)species;

    // molecules of the species in the owned layers
    std::vector<int32_t> hv;
    std::vector<uint32_t> hid;
    std::vector<uint64_t> himg;
    for (int64_t x = 0; x < n; ++x) {
        const int32_t i = ijk[3 * x], j = ijk[3 * x + 1], k = ijk[3 * x + 2];
        if (k < a.k0 || k >= a.k0 + m) continue;
        // wrap counters from the unwrapped position (X = 2I + P, Y = 3J + (K & 1), Z = K)
        const int32_t K = xyz[3 * x + 2];
        const int32_t J = (xyz[3 * x + 1] - (K & 1)) / 3;
        const int32_t I = (xyz[3 * x] - ((J + K) & 1)) / 2;
        const int32_t wi = (I - i) / L->ni, wj = (J - j) / L->nj, wk = (K - k) / L->nk;
        hv.push_back((int32_t)((uint32_t)i + (uint32_t)L->ni * ((uint32_t)j + (uint32_t)L->nj * (uint32_t)(k - a.k0 + 1))));
        hid.push_back(ids[x]);
        himg.push_back((uint64_t)(uint16_t)wi | ((uint64_t)(uint16_t)wj << 16) | ((uint64_t)(uint16_t)wk << 32));
    }
    const int64_t own_n = (int64_t)hv.size();
    const int64_t cap64 = own_n + std::max<int64_t>(own_n / 2, 65536);
    if (cap64 > INT32_MAX / 2) {
        psc_slab_destroy(S);
        return PSC_E_CAPACITY;
    }
    a.cap = (int32_t)cap64;
    a.tcap = (int32_t)std::min<int64_t>((int64_t)nij, std::max<int64_t>(4096, (int64_t)nij / 8));

    // occupancy bits of layers 0 .. m + 1: any species; ghost layers behind a
    // reflective k wall are all ones
    std::vector<uint32_t> hb((size_t)(m + 2) * a.lw, 0u);
    for (int L2 = 0; L2 < m + 2; ++L2) {
        int k = a.k0 - 1 + L2;
        if (k < 0 || k >= L->nk) {
            if (!kper) {
                for (uint32_t w = 0; w < a.lw; ++w) hb[(size_t)L2 * a.lw + w] = ~0u;
                continue;
            }
            k = (k + L->nk) % L->nk;
        }
        for (uint32_t b = 0; b < nij; ++b)
            if (occ[(size_t)k * nij + b]) hb[(size_t)L2 * a.lw + (b >> 5)] |= 1u << (b & 31u);
    }

    S->claim_bytes = 2 * (size_t)nij * 4;
    S->commit_bytes = 8 + (size_t)a.tcap * sizeof(SlabEntry) + (size_t)a.lw * 4;
    a.bits = (uint32_t*)slab_alloc(S, hb.size() * 4);
    a.claim = (uint32_t*)slab_alloc(S, (size_t)(m + 2) * nij * 4);
    for (int x = 0; x < 2; ++x) {
        a.vox[x] = (int32_t*)slab_alloc(S, (size_t)a.cap * 4);
        a.ids[x] = (uint32_t*)slab_alloc(S, (size_t)a.cap * 4);
        a.img[x] = (uint64_t*)slab_alloc(S, (size_t)a.cap * 8);
    }
    a.dec = (uint8_t*)slab_alloc(S, (size_t)a.cap);
    a.count = (int32_t*)slab_alloc(S, 8);
    a.err = (int32_t*)slab_alloc(S, 4);
    for (int x = 0; x < 8; ++x) S->own[x] = slab_alloc(S, x < 4 ? S->claim_bytes : S->commit_bytes);
    for (void* p : S->allocs)
        if (!p) {
            psc_slab_destroy(S);
            return PSC_E_NOMEM;
        }
    S->buf.send_claim[0] = S->own[0]; S->buf.send_claim[1] = S->own[1];
    S->buf.recv_claim[0] = S->own[2]; S->buf.recv_claim[1] = S->own[3];
    S->buf.send_commit[0] = S->own[4]; S->buf.send_commit[1] = S->own[5];
    S->buf.recv_commit[0] = S->own[6]; S->buf.recv_commit[1] = S->own[7];
    bind(S);
    cudaStream_t st = S->stream;
    int32_t counts[2] = {(int32_t)own_n, 0};
    cudaError_t e = cudaMemcpyAsync(a.bits, hb.data(), hb.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.claim, 0xFF, (size_t)(m + 2) * nij * 4, st);
    if (e == cudaSuccess && own_n > 0) e = cudaMemcpyAsync(a.vox[0], hv.data(), (size_t)own_n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && own_n > 0) e = cudaMemcpyAsync(a.ids[0], hid.data(), (size_t)own_n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && own_n > 0) e = cudaMemcpyAsync(a.img[0], himg.data(), (size_t)own_n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.count, counts, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.err, 0, 4, st);
    for (int x = 0; x < 8 && e == cudaSuccess; ++x)
        e = cudaMemsetAsync(S->own[x], 0, x < 4 ? S->claim_bytes : S->commit_bytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        psc_slab_destroy(S);
        return PSC_E_CUDA;
    }
    a.cur = 0;
    *out = S;
    return PSC_OK;
}

extern "C" int psc_slab_buffers_get(const psc_slab* S, psc_slab_buffers* b, int64_t* claim_bytes,
                                    int64_t* commit_bytes)
{
    if (!S || !b || !claim_bytes || !commit_bytes) return PSC_E_ARG;
    *b = S->buf;
    *claim_bytes = (int64_t)S->claim_bytes;
    *commit_bytes = (int64_t)S->commit_bytes;
    return PSC_OK;
}

extern "C" int psc_slab_buffers_set(psc_slab* S, const psc_slab_buffers* b)
{
    if (!S || !b) return PSC_E_ARG;
    for (int side = 0; side < 2; ++side)
        if (!b->send_claim[side] || !b->recv_claim[side] || !b->send_commit[side] || !b->recv_commit[side])
            return PSC_E_ARG;
    S->buf = *b;
    bind(S);
    return PSC_OK;
}

extern "C" int psc_slab_claim(psc_slab* S)
{
    if (!S) return PSC_E_ARG;
    if (S->sticky) return S->sticky;
    if (S->g == UINT32_MAX) return PSC_E_LIMIT;
    DevGuard dg(S->device);
    SlabArgs& a = S->a;
    a.g = S->g;
    const uint32_t nij = (uint32_t)a.ni * (uint32_t)a.nj;
    launch_slab_claim(a, slab_blocks(S, a.cap), S->stream);
    // claim words of layers 0, 1 (to the lower neighbour) and m, m + 1 (to the upper one)
    cudaError_t e = cudaMemcpyAsync(S->buf.send_claim[0], a.claim, S->claim_bytes, cudaMemcpyDeviceToDevice,
                                    S->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(S->buf.send_claim[1], a.claim + (size_t)a.m * nij, S->claim_bytes,
                            cudaMemcpyDeviceToDevice, S->stream);
    if (e == cudaSuccess) e = cudaPeekAtLastError();
    return slab_fail(S, e);
}

extern "C" int psc_slab_commit(psc_slab* S)
{
    if (!S) return PSC_E_ARG;
    if (S->sticky) return S->sticky;
    DevGuard dg(S->device);
    SlabArgs& a = S->a;
    const int work = (int)std::max<int64_t>((int64_t)a.cap, 4 * (int64_t)a.ni * a.nj);
    launch_slab_commit(a, slab_blocks(S, work), S->stream);
    return slab_fail(S, cudaPeekAtLastError());
}

extern "C" int psc_slab_apply(psc_slab* S)
{
    if (!S) return PSC_E_ARG;
    if (S->sticky) return S->sticky;
    DevGuard dg(S->device);
    SlabArgs& a = S->a;
    launch_slab_apply(a, slab_blocks(S, std::max<int64_t>(a.tcap, 2 * (int64_t)a.lw)), S->stream);
    a.cur ^= 1;
    S->g += 1;
    return slab_fail(S, cudaPeekAtLastError());
}

// Events of a set of slabs in one process: the exchanges are device copies
// between the slabs' own buffers (peer copies between devices), ordered by
// CUDA events when the slabs' streams differ.
extern "C" int psc_slabs_run_events(psc_slab** slabs, int32_t count, int64_t n_events)
{
    if (!slabs || count < 1 || n_events < 0) return PSC_E_ARG;
    for (int s = 0; s < count; ++s) {
        if (!slabs[s] || slabs[s]->count != count || slabs[s]->index != s) return PSC_E_ARG;
        if (slabs[s]->sticky) return slabs[s]->sticky;
    }
    const bool kper = (slabs[0]->a.bflags & PSC_PERIODIC_K) != 0;
    std::vector<cudaEvent_t> ev((size_t)count, nullptr);
    for (int s = 0; s < count; ++s) {
        DevGuard dg(slabs[s]->device);
        if (cudaEventCreateWithFlags(&ev[s], cudaEventDisableTiming) != cudaSuccess) {
            for (int q = 0; q < s; ++q) cudaEventDestroy(ev[q]);
            return PSC_E_CUDA;
        }
    }
    auto nb = [&](int s, int side) -> int {      // neighbour on side 0 (below) or 1 (above), -1 at a wall
        int q = side == 0 ? s - 1 : s + 1;
        if (q < 0 || q >= count) {
            if (!kper) return -1;
            q = (q + count) % count;
        }
        return q;
    };
    // receiver r takes from sender q: r's recv[side] <- q's send[1 - side]
    auto exchange = [&](bool claims) -> int {
        for (int s = 0; s < count; ++s) {
            DevGuard dg(slabs[s]->device);
            if (cudaEventRecord(ev[s], slabs[s]->stream) != cudaSuccess) return PSC_E_CUDA;
        }
        for (int r = 0; r < count; ++r) {
            psc_slab* R = slabs[r];
            DevGuard dg(R->device);
            for (int side = 0; side < 2; ++side) {
                const int q = nb(r, side);
                if (q < 0) continue;
                psc_slab* Q = slabs[q];
                if (Q->stream != R->stream && cudaStreamWaitEvent(R->stream, ev[q], 0) != cudaSuccess)
                    return PSC_E_CUDA;
                void* dst = claims ? R->buf.recv_claim[side] : R->buf.recv_commit[side];
                const void* src = claims ? Q->buf.send_claim[1 - side] : Q->buf.send_commit[1 - side];
                const size_t bytes = claims ? R->claim_bytes : R->commit_bytes;
                cudaError_t e = Q->device == R->device
                                    ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, R->stream)
                                    : cudaMemcpyPeerAsync(dst, R->device, src, Q->device, bytes, R->stream);
                if (e != cudaSuccess) return PSC_E_CUDA;
            }
        }
        // a sender's buffers are written again only after its receivers copied them
        for (int r = 0; r < count; ++r) {
            DevGuard dg(slabs[r]->device);
            if (cudaEventRecord(ev[r], slabs[r]->stream) != cudaSuccess) return PSC_E_CUDA;
        }
        for (int s = 0; s < count; ++s)
            for (int side = 0; side < 2; ++side) {
                const int q = nb(s, side);
                if (q < 0 || slabs[q]->stream == slabs[s]->stream) continue;
                DevGuard dg(slabs[s]->device);
                if (cudaStreamWaitEvent(slabs[s]->stream, ev[q], 0) != cudaSuccess) return PSC_E_CUDA;
            }
        return PSC_OK;
    };
    int rc = PSC_OK;
    for (int64_t e = 0; e < n_events && !rc; ++e) {
        for (int s = 0; s < count && !rc; ++s) rc = psc_slab_claim(slabs[s]);
        if (!rc) rc = exchange(true);
        for (int s = 0; s < count && !rc; ++s) rc = psc_slab_commit(slabs[s]);
        if (!rc) rc = exchange(false);
        for (int s = 0; s < count && !rc; ++s) rc = psc_slab_apply(slabs[s]);
    }
    for (int s = 0; s < count; ++s) {
        DevGuard dg(slabs[s]->device);
        cudaEventDestroy(ev[s]);
    }
    return rc;
}

extern "C" int psc_slab_synchronize(psc_slab* S)
{
    if (!S) return PSC_E_ARG;
    DevGuard dg(S->device);
    return check(S);
}

// Molecules of the slab: global (i, j, k), ids and unwrapped positions in the
// basis of psc_unwrapped, in list order.  cap < *n_out: nothing written, E_ARG.
extern "C" int psc_slab_coords(psc_slab* S, int32_t* ijk, uint32_t* ids, int32_t* xyz, int64_t cap, int64_t* n_out)
{
    if (!S || !n_out) return PSC_E_ARG;
    DevGuard dg(S->device);
    int rc = check(S);
    if (rc) return rc;
    const SlabArgs& a = S->a;
    int32_t counts[2] = {0, 0};
    cudaError_t e = cudaMemcpy(counts, a.count, 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return slab_fail(S, e);
    const int64_t n = std::min<int64_t>(counts[a.cur], a.cap);
    *n_out = n;
    if (!ijk || cap <= 0) return PSC_OK;
    if (cap < n) return PSC_E_ARG;
    std::vector<int32_t> v((size_t)std::max<int64_t>(1, n));
    std::vector<uint32_t> id((size_t)std::max<int64_t>(1, n));
    std::vector<uint64_t> w((size_t)std::max<int64_t>(1, n));
    if (n > 0) {
        e = cudaMemcpy(v.data(), a.vox[a.cur], (size_t)n * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(id.data(), a.ids[a.cur], (size_t)n * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(w.data(), a.img[a.cur], (size_t)n * 8, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return slab_fail(S, e);
    }
    const uint32_t nij = (uint32_t)a.ni * (uint32_t)a.nj;
    for (int64_t x = 0; x < n; ++x) {
        const uint32_t lv = (uint32_t)v[x];
        const int32_t L = (int32_t)(lv / nij), r = (int32_t)(lv - (uint32_t)L * nij);
        const int32_t j = r / a.ni, i = r - j * a.ni, k = a.k0 - 1 + L;
        ijk[3 * x] = i; ijk[3 * x + 1] = j; ijk[3 * x + 2] = k;
        if (ids) ids[x] = id[x];
        if (xyz) {
            const int32_t I = i + (int32_t)(int16_t)(w[x] & 0xFFFF) * a.ni;
            const int32_t J = j + (int32_t)(int16_t)((w[x] >> 16) & 0xFFFF) * a.nj;
            const int32_t K = k + (int32_t)(int16_t)((w[x] >> 32) & 0xFFFF) * a.nk;
            xyz[3 * x] = 2 * I + ((J + K) & 1);
            xyz[3 * x + 1] = 3 * J + (K & 1);
            xyz[3 * x + 2] = K;
        }
    }
    return PSC_OK;
}

extern "C" int psc_slab_event_index(const psc_slab* S, uint32_t* g)
{
    if (!S || !g) return PSC_E_ARG;
    *g = S->g;
    return PSC_OK;
}

extern "C" void psc_slab_destroy(psc_slab* S)
{
    if (!S) return;
    DevGuard dg(S->device);
    if (S->stream) cudaStreamSynchronize(S->stream);
    for (void* p : S->allocs)
        if (p) cudaFree(p);
    if (S->own_stream && S->stream) cudaStreamDestroy(S->stream);
    delete S;
}
