// psc_static.cu -- psc_hop_events_static: diffusion events of one species on
// buffers the caller owns, with all scratch in fixed-size device arrays of
// this file, so the call itself never allocates memory.
//
// Who needs it: code that cannot call cudaMalloc at the point where it wants
// to step molecules -- e.g. a host that hands the library pre-registered or
// pooled device memory and forbids further allocation, code running while an
// allocator lock is held, or callers that must avoid the implicit device
// synchronisation cudaMalloc/cudaFree can cause.  Everything such a caller
// cannot provide (claim words, vacancy mirror, counters) lives in the static
// arrays below; every GPU that loads the library holds them until the
// process exits.
#include "psc.h"
#include "psc_internal.h"

#include <mutex>

namespace psc {

// Largest lattice the static scratch serves: 2^21 voxels (e.g. 128^3), with a
// vacancy mirror of at most 2^20 words.  Scratch: 8 MiB of claim words,
// 4 MiB of mirror words, one Scalars block.
constexpr int64_t kStaticMaxVoxels = (int64_t)1 << 21;
constexpr int64_t kStaticMaxMirrorWords = (int64_t)1 << 20;

static __device__ __align__(256) uint32_t g_static_claim[kStaticMaxVoxels];
static __device__ __align__(256) uint32_t g_static_mirror[kStaticMaxMirrorWords];
static __device__ __align__(256) Scalars g_static_scalars;

namespace {

struct StaticDevice {
    bool ready = false;
    uint32_t* claim = nullptr;   // device addresses of the arrays above
    uint32_t* mirror = nullptr;
    Scalars* scalars = nullptr;
    int sm_count = 0;
};

constexpr int kStaticMaxDevices = 64;
StaticDevice g_static_dev[kStaticMaxDevices];
std::mutex g_static_mu;

// Once per device, with that device current: the host-side names of the
// arrays are stand-ins, so their device addresses come from the runtime.
int static_setup(int dev, StaticDevice** out)
{
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticDevice& d = g_static_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_claim) != cudaSuccess || !p) return PSC_E_CUDA;
        d.claim = static_cast<uint32_t*>(p);
        if (cudaGetSymbolAddress(&p, g_static_mirror) != cudaSuccess || !p) return PSC_E_CUDA;
        d.mirror = static_cast<uint32_t*>(p);
        if (cudaGetSymbolAddress(&p, g_static_scalars) != cudaSuccess || !p) return PSC_E_CUDA;
        d.scalars = static_cast<Scalars*>(p);
        if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return PSC_E_CUDA;
        d.ready = true;
    }
    *out = &d;
    return PSC_OK;
}

// every call starts from clean scratch: counters zeroed, the molecule count set
__global__ void k_static_reset(int32_t n)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxSpecies; ++s) {
            g_static_scalars.counts[s] = 0;
            g_static_scalars.tmp_count[s] = 0;
        }
        g_static_scalars.counts[0] = n;
        g_static_scalars.next_id = 0;
        g_static_scalars.births = 0;
        g_static_scalars.err = 0;
        for (int x = 0; x < kNumStats; ++x) g_static_scalars.stats[x] = 0ull;
    }
}

// after the checked mirror build: a call whose molecules failed the checks
// runs its events over zero molecules, so the caller's buffers stay as they were
__global__ void k_static_gate()
{
    if (threadIdx.x == 0 && g_static_scalars.err != 0) g_static_scalars.counts[0] = 0;
}

}  // namespace
}  // namespace psc

using namespace psc;

extern "C" int psc_hop_events_static(int32_t ni, int32_t nj, int32_t nk, uint32_t boundary_flags,
                                     uint64_t seed, int32_t species, uint32_t first_event, int32_t n_events,
                                     int32_t* vox, const uint32_t* ids, uint64_t* img, int32_t n, void* stream)
{
    if (!vox || !ids || !img || n < 0 || n_events < 0 || species < 0 || species >= kMaxSpecies ||
        boundary_flags > 7u)
        return PSC_E_ARG;
    if (ni < 1 || nj < 1 || nk < 1) return PSC_E_DIMS;
    if ((boundary_flags & PSC_PERIODIC_I) && ni < 3) return PSC_E_DIMS;
    if ((boundary_flags & PSC_PERIODIC_J) && (nj < 4 || (nj & 1))) return PSC_E_DIMS;
    if ((boundary_flags & PSC_PERIODIC_K) && (nk < 4 || (nk & 1))) return PSC_E_DIMS;
    const int64_t V = (int64_t)ni * nj * nk;
    const int64_t words = (int64_t)mirror_words(ni, nj, nk);
    if (V > kStaticMaxVoxels || words > kStaticMaxMirrorWords) return PSC_E_CAPACITY;
    if (n > V) return PSC_E_FULL;
    if ((uint64_t)first_event + (uint64_t)n_events > (uint64_t)UINT32_MAX) return PSC_E_LIMIT;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) return PSC_E_CUDA;
    StaticDevice* sd = nullptr;
    int rc = static_setup(dev, &sd);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    Geometry geo{};
    geo.ni = ni; geo.nj = nj; geo.nk = nk; geo.bflags = boundary_flags;
    geo.ninj = (uint32_t)ni * (uint32_t)nj;
    geo.div_ni = make_fastdiv((uint32_t)ni);
    geo.div_ninj = make_fastdiv(geo.ninj);
    geo.nbi = (uint32_t)((ni + 3) / 4);
    geo.nbj = (uint32_t)((nj + 3) / 4);

    // the arrays keep whatever the previous call left: start from a clean state
    const int fill_blocks = sd->sm_count * 4;
    launch_fill_u32(sd->claim, kNoClaim, (size_t)V, fill_blocks, st);
    launch_fill_u32(sd->mirror, 0u, (size_t)words, fill_blocks, st);
    k_static_reset<<<1, 32, 0, st>>>(n);
    SpeciesList list;
    list.vox = vox;
    list.ids = const_cast<uint32_t*>(ids);
    list.img = img;
    list.cap = n;
    launch_mirror_from_list_checked(sd->mirror, geo, list, &sd->scalars->counts[0], V, &sd->scalars->err,
                                    fill_blocks, st);
    k_static_gate<<<1, 32, 0, st>>>();

    EventArgs a{};
    a.geo = geo;
    a.occ = nullptr;                 // a species without reactions never touches codes
    a.bits = sd->mirror;
    a.ct.direct = sd->claim;
    a.list = list;
    a.count = &sd->scalars->counts[0];
    a.model = nullptr;
    a.sc = sd->scalars;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32);
    a.s = species;
    a.live = 0;
    a.collect_stats = 0;
    const int threads = 256;
    int blocks = (int)((n + threads - 1) / threads);
    blocks = blocks < 1 ? 1 : (blocks > sd->sm_count * 8 ? sd->sm_count * 8 : blocks);
    for (int32_t e = 0; e < n_events; ++e) {
        a.g = first_event + (uint32_t)e;
        launch_claim(a, false, blocks, threads, st);
        launch_commit(a, false, blocks, threads, st);
    }
    if (cudaPeekAtLastError() != cudaSuccess) return PSC_E_CUDA;
    // wait for the events and report what the device raised (a plain copy of
    // one word into host memory: no allocation)
    int32_t err = 0;
    if (cudaMemcpyAsync(&err, &sd->scalars->err, sizeof(err), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PSC_E_CUDA;
    if (err & kErrBadInput) return PSC_E_ARG;
    return err ? PSC_E_CAPACITY : PSC_OK;
}
