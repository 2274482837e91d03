// psc_internal.h -- device-side data layout and launch interfaces of the hop
// engine.  Shared by the CUDA translation units and the host runtime; not part
// of the public ABI (include/psc.h).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace psc {

constexpr int kMaxSpecies = 32;
constexpr int kMaxReactions = 128;
constexpr int kMaxFirstOrder = 8;          // first-order reactions per species
constexpr int kMaxCompartments = 16;
constexpr uint32_t kNoClaim = 0xFFFFFFFFu;  // claim word of an unclaimed voxel
constexpr uint16_t kBlocked = 0xFFFFu;      // occupancy code reserved for walls
constexpr uint32_t kTagEvent = 0u;          // Philox counter word 2 domain tags
constexpr uint32_t kTagPopulate = 1u;

// Error bits raised on the device, read back by psc_synchronize.
constexpr int32_t kErrListOverflow = 1;
constexpr int32_t kErrBirthOverflow = 2;
constexpr int32_t kErrClaimTableFull = 4;
constexpr int32_t kErrBarrierTimeout = 8;
constexpr int32_t kErrBadInput = 16;       // caller-supplied molecules: voxel out of range,
                                            // two on one voxel, or the reserved id

// grid-wide barrier state of the persistent hop kernel: one arrival word whose
// top bit flips each time every block has arrived
struct BarrierState {
    unsigned int arrive;
    unsigned int pad;
};

// n / d for n, d < 2^31 by one high multiply (round-up reciprocal).
struct FastDiv {
    uint32_t d;
    uint32_t m;
    int32_t s;  // -1 marks d == 1
};
FastDiv make_fastdiv(uint32_t d);

struct Geometry {
    int32_t ni, nj, nk;
    uint32_t bflags;      // bit a set: axis a periodic
    uint32_t ninj;
    FastDiv div_ni;
    FastDiv div_ninj;
    uint32_t nbi, nbj;    // vacancy-mirror bricks (4 x 4 x 2 voxels per word) along i, j
    // compact Morton code of a voxel = mort[i] | mort[ni + j] | mort[ni + nj + k]
    // (bits of the three axes interleaved, axes with fewer bits dropping out
    // at the top), mort_bits wide
    const uint32_t* mort;
    uint32_t mort_bits;
    uint32_t slot_map;    // claim-table home slot: 0 hashed voxel index, 1 Morton,
                          // 2 Morton with the low 10 bits permuted
};
// host: spread tables of the compact Morton code (ni + nj + nk words)
void build_morton_tables(int32_t ni, int32_t nj, int32_t nk, uint32_t* out, uint32_t* bits);
// words of the vacancy mirror for an ni x nj x nk lattice
inline uint64_t mirror_words(int32_t ni, int32_t nj, int32_t nk)
{
    return (uint64_t)((ni + 3) / 4) * (uint64_t)((nj + 3) / 4) * (uint64_t)((nk + 1) / 2);
}

// Structure-of-arrays list of the molecules of one species.  img packs three
// 16-bit periodic wrap counters (i at bits 0-15, j at 16-31, k at 32-47).
struct SpeciesList {
    int32_t* vox;
    uint32_t* ids;
    uint64_t* img;
    int32_t cap;
};

struct ReactionDev {
    uint64_t T;           // acceptance threshold (second order), floor(p 2^32)
    int32_t np;           // products
    int32_t p0, p1;       // product species
};

// Model tables, uploaded once at populate and read through a pointer.
struct ModelDev {
    int8_t pair[kMaxSpecies][kMaxSpecies];   // second-order reaction or -1
    ReactionDev rx[kMaxReactions];
    uint64_t T_fire[kMaxSpecies];            // first-order firing threshold
    int32_t n_fo[kMaxSpecies];
    int32_t fo_rx[kMaxSpecies][kMaxFirstOrder];
    uint64_t fo_cum[kMaxSpecies][kMaxFirstOrder];
    SpeciesList lists[kMaxSpecies];
    // Compartments (Sec. 2): one vacancy mirror per compartment, in which the
    // voxels of every other compartment are set for good, so a species tests
    // vacancy-and-own-compartment with one bit of its own mirror
    uint32_t* mirror[kMaxSpecies];           // the mirror of the species' compartment
    uint8_t comp[kMaxSpecies];               // the species' compartment
};

enum StatIndex {
    kStatAttempts = 0, kStatHops, kStatCollisions, kStatAccepted, kStatReactions2,
    kStatFires, kStatReactions1, kStatBirths, kNumStats
};

// Small device-resident scalars of one lattice.
struct Scalars {
    int32_t counts[kMaxSpecies];     // molecules per species list
    int32_t tmp_count[kMaxSpecies];  // entries of each list that left in the current event
    uint32_t next_id;                // next fresh molecule id
    int32_t births;                  // births queued in the current event
    int32_t err;                     // kErr* bits
    uint32_t g_base;                 // index of the first event of a replayed graph
    unsigned long long stats[kNumStats];
};

struct Birth {
    uint32_t parent;
    int32_t t;
    int32_t species;
    int32_t pad;
    uint64_t img;
};

// Where the claims of one event go.  Direct: one 32-bit word per voxel (small
// lattices), reset by the winner.  Hash: open addressing over 64-bit slots
// holding (voxel << 32 | lowest id); two tables alternate between events and
// the commit kernel of one event empties the table of the previous one.
struct ClaimTable {
    uint32_t* direct;
    uint64_t* hash;
    uint32_t hash_bits;        // log2 of the slots in use this event
    uint64_t* clear;           // table of the previous event (hash mode)
    uint32_t clear_n;          // its slots to reset
};
constexpr uint64_t kEmptySlot = ~0ull;

// Everything one event kernel needs, passed by value.
struct EventArgs {
    Geometry geo;
    uint16_t* occ;             // species codes (exact for species with reactions)
    uint32_t* bits;            // vacancy mirror: bit v set = voxel v occupied
    ClaimTable ct;
    SpeciesList list;          // list of the due species
    const int32_t* count;      // its length (device)
    const ModelDev* model;
    Scalars* sc;
    Birth* births;
    int32_t births_cap;
    uint32_t key0, key1;       // Philox key = seed
    uint32_t g;                // global event index (with g_base: its offset from *g_base)
    const uint32_t* g_base;    // null, or the device word holding the index a replayed graph starts at
    uint32_t* dirty[2];        // by event parity: a bit per mirror word whose voxels changed species
    uint32_t dirty_words;      // words of one dirty map
    uint8_t* dec;              // null, or per list entry the claim's outcome for the commit (kDec*)
    int32_t* leave;            // species with reactions: the commit notes here the slots of the due
                               // species' entries that react away (count in Scalars::tmp_count[s])
    uint32_t* g_bump;          // null, or the word the event's last launch sets to its index + 1
    int32_t* holes;            // scratch of the own-list fill of a one-block event (the scratch
    int32_t* surv;             // list's ids and img; img's decision bytes are read by then)
    int32_t s;                 // due species
    int32_t live;              // 1: the species writes its code into occ
    int32_t collect_stats;
};

// Outcome of a molecule's claim phase, kept for its commit phase: the
// direction 0-11 of the voxel it claimed, no claim, or a first-order firing
// (the commit redraws those)
constexpr uint8_t kDecNone = 12;
constexpr uint8_t kDecFire = 13;

// A stretch of consecutive events of one species without reactions, run by
// one persistent cooperative launch.
struct RunArgs {
    EventArgs ev;              // g = index of the first event
    uint64_t* tables[2];       // claim tables, alternating by event parity
    int32_t n_events;
    BarrierState* barrier;
    uint64_t barrier_timeout_ns;  // a block gives up waiting at a barrier after this long
    uint32_t barrier_phantom;     // arrivals awaited from blocks that do not exist (0; tests only)
};

// Owner-computes decomposition of a stretch (tile kernel): the mirror's brick
// grid (nbi x nbj x nbk words) is cut into pi x pj x pk boxes of whole bricks,
// one per block; region a along an axis of nb bricks spans bricks
// [a nb / p, (a + 1) nb / p).
struct TilePlan {
    int32_t pi, pj, pk;
    int32_t nbi, nbj, nbk;
    int32_t ei, ej, ek;        // largest region extent in bricks
    int32_t regions;
    int32_t box_words;         // (ei + 2)(ej + 2)(ek + 2): region plus one brick of halo
    int32_t cap;               // molecule slots per region (bucket, inbox)
    int32_t fcc;               // FCC lattice: stencil and neighbourhood masks by k mod 3
    int32_t lean;              // 1: the stretch runs k_tile_lean (HCP, whole bricks, boxes of
                               // at least two bricks, two or more boxes along periodic axes)
};

// A stretch of a species without reactions under the tile kernel.  Each
// region's molecules live in its bucket; a molecule that hops into another
// region is appended to that region's inbox and joins its bucket at the next
// event.  Wrap counters are kept by id (the species' ids are id_lo .. id_lo +
// n - 1: it never reacts, so they are the ones populate gave it).
struct TileArgs {
    EventArgs ev;              // g = index of the first event
    TilePlan plan;
    uint32_t* claim;           // per-voxel claim words (kNoClaim when free), for contested targets
    uint32_t* claimed;         // [regions] events whose claim phase the region has finished
    uint32_t* done;            // [regions] events whose commit phase the region has finished
    int32_t nbr_sync;          // 1: phases wait for the neighbouring boxes only; 0: grid barriers
    int32_t* b_vox[2];         // [regions][cap] voxel of each molecule; event e
    uint32_t* b_ids[2];        // reads buffer e & 1 and keeps its survivors in the other
    uint32_t* b_state;         // claim-phase decision of each bucket slot
    int32_t* b_cnt;            // [regions]
    int32_t* in_vox;           // [regions][cap] arrivals of the last event
    uint32_t* in_ids;
    int32_t* in_cnt;           // [regions]
    uint64_t* img_id;          // wrap counters by id - id_lo
    uint2* halo_tab;           // lean kernel: [regions][halo_cap] (box word, global word or ~0 behind a wall)
    int32_t halo_cap;
    uint32_t id_lo;
    int32_t n_events;
    BarrierState* barrier;
    uint64_t barrier_timeout_ns;
    uint32_t barrier_phantom;
};

// A stretch of events of one species under the sub-volume rule (the paper's
// sub-volume scheme on the lattice; species without reactions).
struct SubvolArgs {
    EventArgs ev;              // g = index of the first event
    uint32_t* word;            // per 2x2x2 sub-volume: lowest waiting id of the colour's turn (kNoClaim: free)
    uint32_t* head;            // per sub-volume: first list slot of its chain of waiting molecules (kNoClaim: none)
    uint32_t* next;            // per list slot: the next slot of its sub-volume's chain
    uint32_t* state;           // per list slot: its sub-volume at the event's start, bit 31 it leads it, bit 30 alone
    uint8_t* colour0;          // per list slot: colour of its sub-volume when the event began
    uint32_t* lead;            // per list slot: the leaders' slots, colour by colour (top bit: alone)
    uint32_t* lead_vox;        // per list slot: the voxel of an alone leader, in the same order
    uint32_t* counters;        // [2][16] by event parity: molecules and leaders per colour
    int32_t n_events;
    BarrierState* barrier;
    uint64_t barrier_timeout_ns;
    uint32_t barrier_phantom;
};

struct ReconcileArgs {
    Geometry geo;
    uint16_t* occ;
    const uint32_t* bits;
    int32_t x;                 // species whose list is reconciled
    SpeciesList list;
    SpeciesList tmp;           // scratch: the slots that leave, then the holes and the tail's survivors
                               // (vox and ids hold twice the capacity: one reaction can remove two entries)
    const ModelDev* model;
    Scalars* sc;
    const uint32_t* dirty[2];  // the commit's dirty maps, by event parity
    uint32_t g;                // event index (with g_base: its offset from *g_base)
    const uint32_t* g_base;
    uint32_t* g_bump;          // null, or the word the event's last launch sets to its index + 1
};

// ---- launchers (psc_kernels.cu) ----
void upload_stencil(cudaStream_t st);
void launch_claim(const EventArgs& a, bool general, int blocks, int threads, cudaStream_t st);
void launch_commit(const EventArgs& a, bool general, int blocks, int threads, cudaStream_t st);
// claim, commit and the own-list fill of one event of a species with
// reactions in a single block (lists of a few hundred molecules)
constexpr int kEventOneThreads = 512;
void launch_event_one(const EventArgs& a, cudaStream_t st);
void launch_fill_u64(uint64_t* p, uint64_t value, size_t n, int blocks, cudaStream_t st);
// Molecules per thread the persistent kernel holds in registers (0 = the
// stretch does not fit); threads = its launch width.
int run_capacity(int64_t n, int* threads_per_block, int* blocks, int sm_count, int min_per_thread);
cudaError_t launch_run(const RunArgs& r, int blocks, int threads, int per_thread, cudaStream_t st);
cudaError_t launch_subvol(const SubvolArgs& A, int blocks, int threads, cudaStream_t st);
int subvol_max_blocks(int sm_count);        // co-resident 256-thread blocks of the sub-volume kernel
// tile kernel: dynamic shared memory a block may use, its need for a plan,
// the three launches of a stretch (list -> buckets, the persistent events,
// buckets -> list)
int tile_smem_limit(int device);
constexpr int kTileOutbox = 1024;           // departures a block stages per event
constexpr int kTileQueue = 1024;            // molecules a block defers per commit phase (contested, leaving)
// largest max / mean box load at which the automatic choice keeps the tile kernel
constexpr double kTileMaxImbalance = 1.4;
inline int tile_smem_bytes(const TilePlan& P)
{
    return ((P.box_words + 3) & ~3) * 4 + (P.fcc ? 96 : 32) * 8 * 4 + kTileOutbox * 12 + kTileQueue * 4 +
           ((P.nbi + P.nbj + P.nbk + 15) & ~15);
}
// the lean tile kernel: shared-memory tables per (place in the brick word,
// direction), per-axis halo tables, plus the areas of the general kernel
constexpr int kLeanEntries = 32 * 12;
constexpr int kLeanClaimBits = 10;          // block-local claim table: 2^10 slots of 8 bytes
constexpr int kLeanOutbox = 512;            // departures staged per event (more go straight to the inboxes)
// halo words of the largest box of a plan (the lean kernel's per-box halo table)
inline int64_t lean_halo_cap(const TilePlan& P)
{
    const int64_t BI = P.ei + 2, BJ = P.ej + 2, BK = P.ek + 2;
    return 2 * BI * BJ + 2 * (BK - 2) * BI + 2 * (BK - 2) * (BJ - 2);
}
inline int lean_smem_bytes(const TilePlan& P)
{
    const int halo_tables = ((P.ei + 2) + (P.ej + 2) + (P.ek + 2) + 3) & ~3;
    return ((P.box_words + 3) & ~3) * 4 + (8 << kLeanClaimBits) + kLeanEntries * 8 * 4 + kLeanEntries * 2 * 4 +
           kLeanOutbox * 12 + halo_tables * 4 + ((P.box_words + 31) >> 5) * 4 +
           ((P.nbi + P.nbj + P.nbk + 15) & ~15);
}
constexpr int kTileThreads = 512;
constexpr int kTileBlocksPerSM = 2;
void launch_tile_count(const TileArgs& A, int32_t* counts, int blocks, cudaStream_t st);
void launch_tile_scatter(const TileArgs& A, int blocks, cudaStream_t st);
cudaError_t launch_tile_run(const TileArgs& A, cudaStream_t st);
void launch_tile_gather(const TileArgs& A, cudaStream_t st);
// mirror c of n: bit v set where labels[v] != c (walls), the rest clear
void launch_mirror_walls(uint32_t* bits0, uint64_t words, int n, const uint8_t* labels, const Geometry& geo,
                         int blocks, cudaStream_t st);
// placement by selection (psc_populate): per compartment, a histogram of the
// top kPlaceBits bits of the voxels' placement keys, then the voxels whose
// key bin is at most that compartment's limit (-1: none), in no order
constexpr int kPlaceBits = 10;
struct PlaceLimits {
    int32_t bin[kMaxCompartments];
};
void launch_place_hist(uint32_t V, uint32_t key0, uint32_t key1, const uint8_t* labels, int nc, uint32_t* hist,
                       int blocks, cudaStream_t st);
void launch_place_pick(uint32_t V, uint32_t key0, uint32_t key1, const uint8_t* labels, const PlaceLimits& lim,
                       uint32_t* out_vox, uint32_t* out_key, int32_t* count, int32_t cap, int32_t* err, int blocks,
                       cudaStream_t st);
// keys[r] = labels[vals[r]]: the compartment of each sorted voxel
void launch_label_keys(const uint32_t* vals, const uint8_t* labels, uint32_t* keys, int64_t n, int blocks,
                       cudaStream_t st);
// codes where a voxel is occupied (its bit set in all n_mirrors mirrors of
// `words` words each, starting at bits0), zero elsewhere
void launch_materialize(uint16_t* out, const uint16_t* occ, const uint32_t* bits0, uint64_t words,
                        int n_mirrors, const Geometry& geo, int64_t V, int blocks, cudaStream_t st);
void launch_scatter_codes(uint16_t* out, const SpeciesList& list, const int32_t* count, uint16_t code,
                          int blocks, cudaStream_t st);
// Partner list r.x checked against the grid; its leavers' slots go after
// those of the lists in `before` (a bit per species).
void launch_reconcile(const ReconcileArgs& r, uint32_t before, int blocks, int threads, cudaStream_t st);
// The event's lists filled from their tails, one block each, side by side.
constexpr int kListFillMax = 8;
struct ListFill {
    ReconcileArgs r;                       // the event's arguments; x and list per block
    int32_t n;
    int32_t x[kListFillMax];
    SpeciesList list[kListFillMax];
    uint32_t before[kListFillMax];         // lists whose scratch ranges come first
};
void launch_fill(const ListFill& f, cudaStream_t st);
void launch_births(const EventArgs& a, cudaStream_t st);
void launch_fill_u32(uint32_t* p, uint32_t value, size_t n, int blocks, cudaStream_t st);
// molecule r (ids in species order, species s owning [offsets[s],
// offsets[s+1])) takes sorted_vox[starts[s] + r - offsets[s]]; its bit goes
// to the mirror of its species' compartment
void launch_populate_scatter(const uint32_t* sorted_vox, int64_t n_total, const int64_t* offsets,
                             const int64_t* starts, int n_species, uint16_t* occ, const Geometry& geo,
                             const ModelDev* model, int blocks, cudaStream_t st);
// The Morton re-sort of a list's first min(*count, limit) entries (the rest,
// if any, keep their places: list order never changes results).
void launch_morton_keys(const SpeciesList& list, const int32_t* count, int32_t limit, const Geometry& geo,
                        uint32_t* keys, uint32_t* vals, int blocks, cudaStream_t st);
uint32_t morton_sort_bits(const Geometry& geo);
void launch_permute(const SpeciesList& src, const SpeciesList& dst, const uint32_t* perm,
                    const int32_t* count, int32_t limit, int blocks, cudaStream_t st);
void launch_copy_list(const SpeciesList& src, const SpeciesList& dst, const int32_t* count, int32_t limit,
                      int blocks, cudaStream_t st);
// set the vacancy-mirror bit of every molecule of a list (mirror cleared before)
void launch_mirror_from_list(uint32_t* bits, const Geometry& geo, const SpeciesList& list, const int32_t* count,
                             int blocks, cudaStream_t st);
// the same for a list the library did not build: entries whose voxel is
// outside [0, V), that land on a voxel already set, or whose id is kNoClaim
// are skipped and raise kErrBadInput in *err
void launch_mirror_from_list_checked(uint32_t* bits, const Geometry& geo, const SpeciesList& list,
                                     const int32_t* count, int64_t V, int32_t* err, int blocks, cudaStream_t st);

// ---- slabs along k with ghost layers (psc_slab.cuh, psc_slab.cpp) ----
struct SlabEntry {                 // a molecule handed to a neighbouring slab
    int32_t i, j, k;               // global coordinates of the voxel it entered
    uint32_t id;
    uint64_t img;                  // packed wrap counters
};

struct SlabArgs {
    int32_t ni, nj, nk, m, k0;     // global extents, owned layers, first owned layer
    uint32_t bflags;
    uint32_t lw;                   // words per layer of the bit array (layers start on words)
    uint32_t* bits;                // (m + 2) * lw words: bit i + ni j of layer L, set = occupied or wall
    uint32_t* claim;               // (m + 2) * ni * nj words, kNoClaim when free
    int32_t* vox[2];               // molecule lists by buffer: local voxel i + ni (j + nj L)
    uint32_t* ids[2];
    uint64_t* img[2];
    int32_t* count;                // [2] molecules per buffer
    int32_t cap;
    int32_t cur;                   // buffer holding the molecules at the start of the event
    uint8_t* dec;                  // claim-phase decision per molecule
    uint8_t* send_commit[2];       // [0] to the lower neighbour, [1] to the upper one
    const uint8_t* recv_commit[2];
    const uint32_t* recv_claim[2];
    int32_t tcap;                  // entries a commit message holds
    int32_t has[2];                // a neighbour on that side (else a wall)
    int32_t* err;
    uint32_t key0, key1, g, s;     // Philox key, event index, species
};

void launch_slab_claim(const SlabArgs& A, int blocks, cudaStream_t st);
void launch_slab_commit(const SlabArgs& A, int blocks, cudaStream_t st);
void launch_slab_apply(const SlabArgs& A, int blocks, cudaStream_t st);

// ---- batched launches: many lattices (replicas) per launch ----
// Item x covers blocks [block0, next block0) of the launch and runs the event
// (or list) `sel` of replica `rep` with event index g.  Argument templates of
// every (replica, species) live on the device: tmpl[rep * kMaxSpecies + sel].
constexpr int kBatchMax = 512;
struct BatchItem {
    int32_t rep;
    int32_t sel;
    uint32_t g;
    int32_t block0;
    uint32_t mask;             // list passes: lists whose scratch ranges come before list sel's
};
struct BatchLaunch {
    int32_t n;
    int32_t total_blocks;
    BatchItem item[kBatchMax];
};
void launch_claim_batch(const EventArgs* tmpl, const BatchLaunch& bl, int threads, cudaStream_t st);
void launch_commit_batch(const EventArgs* tmpl, const BatchLaunch& bl, int threads, cudaStream_t st);
void launch_reconcile_batch(const ReconcileArgs* tmpl, const BatchLaunch& bl, int threads, cudaStream_t st);
void launch_fill_batch(const ReconcileArgs* tmpl, const BatchLaunch& bl, cudaStream_t st);
void launch_births_batch(const EventArgs* tmpl, const BatchLaunch& bl, cudaStream_t st);

// ---- radix sort (psc_sort.cu) ----
// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of key.
// n is n_host, or the count in device memory (n_dev) capped at n_host;
// max_n (at least n_host) sizes the tiles and the scratch.
struct SortScratch {
    uint32_t* keys_alt = nullptr;
    uint32_t* vals_alt = nullptr;
    uint32_t* hist = nullptr;       // 256 * blocks
    uint32_t* block_sums = nullptr; // scan partials
    int64_t max_n = 0;
    int64_t hist_len = 0;
    int64_t sums_len = 0;
};
size_t sort_scratch_bytes(int64_t max_n);
void sort_scratch_bind(SortScratch& s, void* base, int64_t max_n);
// After the call the sorted data is in (keys, vals) again.
int radix_sort_pairs(uint32_t* keys, uint32_t* vals, const int32_t* n_dev, int64_t n_host,
                     int64_t max_n, int bits, SortScratch& scratch, cudaStream_t st,
                     int64_t* launches);

}  // namespace psc
