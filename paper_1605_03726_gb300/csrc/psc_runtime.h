// psc_runtime.h -- host-side lattice state shared by the runtime files
// (psc_api.cpp: single lattices; psc_batch.cpp: batches and the server).
// Not part of the public ABI.
#pragma once

#include "psc.h"
#include "psc_internal.h"

#include <cstdint>
#include <vector>

namespace psc_rt {

using namespace psc;

struct Species {
    double D = 0.0;
    int64_t n0 = 0;
    double tau = 0.0;
    uint64_t done = 0;
    int n_fo = 0;
    int fo[kMaxFirstOrder] = {};
    int comp = 0;                      // compartment (Sec. 2)
};

struct Reaction {
    int nr = 0, np = 0;
    int r[2] = {0, 0}, p[2] = {0, 0};
    double k = 0.0;
    double prob = 0.0;
};

}  // namespace psc_rt

using namespace psc;

struct psc_lattice {
    int32_t ni = 0, nj = 0, nk = 0;
    int64_t V = 0;
    double rv = 0.0;
    uint32_t bflags = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;

    int nsp = 0;
    psc_rt::Species sp[kMaxSpecies];
    int nrx = 0;
    psc_rt::Reaction rx[kMaxReactions];
    int8_t pair[kMaxSpecies][kMaxSpecies];

    bool populated = false;
    bool clamped = false;
    uint64_t seed = 0;
    uint32_t g = 0;
    double clock = 0.0;

    psc::Geometry geo{};
    ModelDev model_h{};
    ModelDev* model_d = nullptr;
    uint16_t* occ = nullptr;
    uint32_t* bits = nullptr;          // vacancy mirrors, one bit per voxel, one mirror per compartment
    uint32_t* dirty[2] = {nullptr, nullptr};   // by event parity: mirror words whose voxels changed species
    uint32_t dirty_words = 0;
    uint64_t mirror_n = 0;             // words of one mirror
    int32_t ncomp = 1;                 // compartments (Sec. 2)
    std::vector<uint8_t> labels;       // compartment of every voxel (empty: all 0)
    uint32_t* claim = nullptr;         // per-voxel claim words (small lattices)
    uint64_t* tables[2] = {nullptr, nullptr};   // claim hash tables (large lattices)
    uint32_t table_used[2] = {0, 0};   // slots written by the event that used it
    int64_t table_slots = 0;
    BarrierState* barrier = nullptr;
    uint32_t hash_bits[kMaxSpecies] = {};
    Scalars* sc = nullptr;
    Birth* births = nullptr;
    int32_t births_cap = 0;
    SpeciesList tmp{};
    int32_t cap[kMaxSpecies] = {};
    uint32_t* rs_keys = nullptr;      // re-sort keys / values
    uint32_t* rs_vals = nullptr;
    SortScratch rs_scratch;
    int64_t rs_max = 0;
    int32_t* readout = nullptr;          // staging of the device-side read-out (16 bytes per molecule)
    int64_t readout_cap = 0;

    bool general[kMaxSpecies] = {};
    // automatic stretch kernel (psc_options.tiles = 0) of species with a tile
    // plan: 0 not decided yet, 1 the tile kernel, -1 the molecule-list kernel
    int8_t tile_auto[kMaxSpecies] = {};
    bool live[kMaxSpecies] = {};       // takes part in a reaction: keeps its codes
    bool fo2[kMaxSpecies] = {};
    std::vector<int> reconcile[kMaxSpecies];
    uint64_t since_resort[kMaxSpecies] = {};

    psc_options opt{64, 256, 8, 0, 32, 0, 0, 1, 1, 3, 0, 1000000, 0, 0, 0, -1, 1};
    int64_t launches = 0;
    uint64_t events = 0;
    uint64_t h2d = 0, d2h = 0;

    // CUDA-event spans around kernels (psc_options.time_kernels)
    struct Span { cudaEvent_t a, b; int kind; int64_t events; };
    std::vector<Span> spans;
    std::vector<cudaEvent_t> event_pool;
    int sticky = PSC_OK;
    std::vector<void*> allocs;

    // per-event runs replayed from CUDA graphs (psc_options.graph_events):
    // graphs by run pattern, patterns seen once, and the first event index
    // of a run being captured (-1: none)
    struct GraphRun {
        std::vector<uint8_t> key;
        cudaGraphExec_t exec = nullptr;
        uint32_t table_used[2] = {0, 0};
        std::vector<uint64_t> since;
        int64_t launches = 0;
    };
    std::vector<GraphRun> graphs;
    std::vector<std::vector<uint8_t>> graph_seen;
    // single events replayed from graphs (runs whose pattern does not recur)
    std::vector<GraphRun> graphs1;
    std::vector<std::vector<uint8_t>> graph_seen1;
    int64_t capture_g0 = -1;
    bool capture_single = false;
    // Host estimates of the list lengths, for the per-event grids only (every
    // per-event kernel strides over the count in device memory, so a stale
    // estimate costs time, never results): a pinned copy of Scalars::counts
    // refreshed in the background every few events.
    int64_t est[kMaxSpecies] = {};
    int32_t grid_class[kMaxSpecies] = {};  // per-event grid limit of each list (INT32_MAX: none)
    int32_t* counts_h = nullptr;
    cudaEvent_t counts_ev = nullptr;
    bool counts_pending = false;
    uint32_t counts_g = 0;       // capturing one event: its last launch advances Scalars::g_base
    int64_t g_dev = -1;                // what Scalars::g_base holds once the queued work is done (-1 unknown)

    // tile kernel buffers (allocated on first use, grown when a plan needs more)
    struct TileBuffers {
        int64_t slots = 0;             // regions x cap
        int32_t regions = 0;
        int64_t ids = 0;               // entries of img_id
        int32_t* b_vox[2] = {nullptr, nullptr};
        uint32_t* b_ids[2] = {nullptr, nullptr};
        uint32_t* b_state = nullptr;
        int32_t* b_cnt = nullptr;
        int32_t* in_vox = nullptr;
        uint32_t* in_ids = nullptr;
        int32_t* in_cnt = nullptr;
        uint32_t* claimed = nullptr;
        uint32_t* done = nullptr;
        uint64_t* img_id = nullptr;
        uint32_t* claim = nullptr;     // per-voxel claim words when the lattice has none
        uint2* halo_tab = nullptr;     // lean kernel: halo word table per box
        int64_t halo_entries = 0;
    } tile;
    int tile_smem = -1;                // shared memory a tile block may use (-1: not queried yet)

    // sub-volume rule buffers (allocated at populate when the rule is on)
    struct SubvolBuffers {
        uint32_t* word = nullptr;
        uint32_t* head = nullptr;
        uint32_t* next = nullptr;
        uint32_t* state = nullptr;
        uint8_t* colour0 = nullptr;
        uint32_t* lead = nullptr;
        uint32_t* lead_vox = nullptr;
        uint32_t* counters = nullptr;
        int64_t subvols = 0, slots = 0;
        int blocks = 0;
    } subvol;
};

namespace psc_rt {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) { cudaGetDevice(&prev); if (prev != dev) cudaSetDevice(dev); }
    ~DevGuard() { int cur = -1; cudaGetDevice(&cur); if (prev >= 0 && cur != prev) cudaSetDevice(prev); }
};

int cuda_fail(psc_lattice* L, cudaError_t e);
void* dev_alloc(psc_lattice* L, size_t bytes);
int event_blocks(const psc_lattice* L, int64_t work);
int list_blocks(const psc_lattice* L, int x);
int32_t sort_limit(const psc_lattice* L, int x);
bool sorted_order_pays(const psc_lattice* L, int x);
EventArgs event_args(const psc_lattice* L, int s);
ReconcileArgs reconcile_args(const psc_lattice* L, int x);
bool next_event(const psc_lattice* L, int* s_out, double* t_out);
int check_device(psc_lattice* L);
// queue events in scheduler order until max_events or the next event lies after t_end
int drive(psc_lattice* L, double t_end, int64_t max_events);
// drop every captured graph (launch options changed)
void graph_cache_clear(psc_lattice* L);
// Morton re-sort of species s's list (queued on the lattice's stream)
int resort(psc_lattice* L, int s);
void dev_free_one(psc_lattice* L, void* p);
// Can stretches of species s run under the tile kernel?  Fills the plan.
bool tile_plan(psc_lattice* L, int s, TilePlan* P);
int enqueue_tiles(psc_lattice* L, int s, int64_t n_events, const TilePlan& P);
int enqueue_subvol(psc_lattice* L, int s, int64_t n_events);

}  // namespace psc_rt
