/*
 * psc.h -- C ABI of the GB300 voxel hop engine (pSpatiocyte's diffusion and
 * collision step on a hexagonal close-packed lattice).
 *
 * Paper: A. Miyauchi, K. Iwamoto, S. N. V. Arjunan, K. Takahashi,
 * "pSpatiocyte: A Parallel Stochastic Method for Particle Reaction-Diffusion
 * Systems", arXiv:1605.03726.
 *
 * Model (what the calls compute)
 *   Lattice     ni x nj x nk voxels of radius r_v on an HCP lattice in twisted
 *               Cartesian coordinates (Sec. 2.1): i is the straight axis, j and
 *               k zigzag; voxel (i, j, k) has 12 neighbours at distance 2 r_v,
 *               chosen by the parity of j + k and of k.  Voxel index
 *               v = i + ni * (j + nj * k).  Each axis is periodic or closed by
 *               a reflective wall (a hop through a wall fails, Sec. 2.3).
 *   Species     diffusion coefficient D; hop interval tau = 2 r_v^2 / (3 D)
 *               (Sec. 2.3, Eq. 3).  D = 0 marks an immobile species.
 *   Event       the scheduler (Sec. 2.2) picks the mobile species with the
 *               earliest next diffusion time (events_done + 1) * tau; ties go to
 *               the lower species index.  In that event every molecule of the
 *               species draws one of its 12 neighbours and moves there if it is
 *               vacant (Sec. 2.3); if the neighbour holds a registered
 *               second-order partner the pair reacts with probability
 *               p_AB = k / (6 sqrt(2) (D_A + D_B) r_v) (Sec. 2.4.2, Eq. 6,
 *               clamped to 1).  A species with first-order reactions first
 *               tests, per molecule, whether one fires (probability
 *               1 - exp(-sum(k) tau), choice by Eq. 5, Sec. 2.4.1); a molecule
 *               that fires does not hop in that event.
 *   Conflicts   all molecules of the due species decide against the grid as
 *               it was when the event began; a voxel wanted by several goes to
 *               the lowest molecule id; a voxel left in the event is free only
 *               from the next event on.  (The paper updates one molecule at a
 *               time, Sec. 2.3, and says the order barely matters; this
 *               deterministic synchronous form is what runs in parallel.)
 *   Products    second order: the first product takes the partner's voxel and
 *               id, the second the mover's voxel and id.  First order: the
 *               first product keeps the reactant's voxel and id; a second
 *               product goes to a uniformly chosen neighbour that was vacant
 *               at the start of the event (Sec. 2.4.1), contested like a hop,
 *               and gets a fresh id; fresh ids within one event go to the
 *               parents in ascending parent id.
 *   Randomness  Philox4x32-10 keyed by the 64-bit seed; counter
 *               (molecule id, event index, species << 4, 0) for the event
 *               draws and (voxel, 0, 1, 0) for placement.  Results are a pure
 *               function of the model and the seed.
 *
 * Ownership and threading
 *   A psc_lattice is opaque and owns all its device memory; the caller owns
 *   every host buffer passed in.  Device memory comes from cudaMalloc unless
 *   psc_set_allocator installed another allocator.  All device work of a
 *   lattice is queued on its CUDA stream; psc_run and psc_run_events return
 *   once the work is queued, and device-side errors surface at the next call
 *   that synchronises (psc_synchronize and every read-out).  One host thread
 *   at a time per lattice; different lattices are independent.
 *
 * Status codes
 *   0 success; negative values are errors (psc_status_string names them);
 *   PSC_W_PCLAMP (positive) is a warning: some p_AB exceeded 1 and was clamped.
 */
#ifndef PSC_H
#define PSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSC_OK               0
#define PSC_E_ARG           -1   /* bad argument (null pointer, bad index, NaN) */
#define PSC_E_DIMS          -2   /* lattice shape not allowed, see create      */
#define PSC_E_ORDER         -3   /* call out of order (e.g. add after populate) */
#define PSC_E_FULL          -4   /* more molecules than voxels                 */
#define PSC_E_UNSUPPORTED   -5   /* model feature outside this engine          */
#define PSC_E_NOMEM         -6   /* device or host allocation failed           */
#define PSC_E_CUDA          -7   /* CUDA runtime error                         */
#define PSC_E_TIMEOUT       -8   /* a bounded device wait gave up              */
#define PSC_E_LIMIT         -9   /* event counter (2^32 - 1 events) exhausted  */
#define PSC_E_CAPACITY     -10   /* a device list overflowed its capacity      */
#define PSC_W_PCLAMP         1   /* p_AB > 1 clamped to 1 (warning)            */

#define PSC_PERIODIC_I  1u       /* boundary flag bits: set = periodic axis,   */
#define PSC_PERIODIC_J  2u       /* clear = reflective wall                    */
#define PSC_PERIODIC_K  4u
#define PSC_PERIODIC_ALL 7u
#define PSC_FCC         8u       /* lattice flag: FCC (ABC stacking of the same
                                    triangular layers, App. B) instead of HCP  */

#define PSC_MAX_SPECIES    32
#define PSC_MAX_REACTIONS 128
#define PSC_MAX_COMPARTMENTS 16

typedef struct psc_lattice psc_lattice;

/* Counters accumulated on the device when statistics are switched on
   (psc_options.collect_stats); attempts counts every molecule processed in an
   event whatever the outcome. */
typedef struct {
    uint64_t attempts, hops, collisions, accepted, reactions2, fires, reactions1, births;
    uint64_t events;          /* species events queued                         */
    uint64_t launches;        /* kernels launched by this lattice (host count) */
    uint64_t h2d_bytes;       /* bytes copied host -> device by the library    */
    uint64_t d2h_bytes;       /* bytes copied device -> host by the library    */
} psc_stats;

/* Device time of the event kernels, measured with CUDA events recorded on the
   lattice's stream around each launch while psc_options.time_kernels is on. */
typedef struct {
    double claim_ms, commit_ms, reconcile_ms, resort_ms;
    int64_t claim_launches, commit_launches, reconcile_events, resorts;
    double run_ms;            /* persistent launches over stretches of events  */
    int64_t run_launches, run_events;
    int64_t tile_launches, tile_events;   /* of those, under the tile kernel   */
    int64_t tile_lean_events;             /* of those, under its lean variant  */
} psc_kernel_times;

/* Tunables; zero in a field keeps the current value. */
typedef struct {
    int32_t resort_period;    /* events of a species between Morton re-sorts of
                                 its molecule list (default 64; <0 = never);
                                 lists holding fewer than 1/256 of the voxels
                                 are not re-sorted (order never changes results) */
    int32_t block_threads;    /* threads per block of the event kernels (256)   */
    int32_t blocks_per_sm;    /* resident blocks per SM for grid sizing (8)     */
    int32_t collect_stats;    /* 1 = count attempts/hops/... (default 0), -1 off */
    int32_t graph_events;     /* >= 2: runs of this many events that take
                                 per-event launches (species with reactions,
                                 or persistent = -1) are captured in a CUDA
                                 graph the second time their pattern (species
                                 in order, claim-table state, re-sort
                                 counters) comes up and replayed from then
                                 on, the event index read from device memory;
                                 same results, fewer launches.  Off while
                                 time_kernels is on; -1 = off (default 32).
                                 A capture takes in everything queued on the
                                 lattice's stream meanwhile: a stream that
                                 other threads also feed needs -1              */
    int32_t time_kernels;     /* 1 = record CUDA events around the kernels of
                                 every event (psc_kernel_times_get), -1 off     */
    int32_t claim_table;      /* before populate: 1 = one claim word per voxel,
                                 2 = hash table of claims, 0/-1 = by size (a
                                 word per voxel up to 2^22 voxels, or where
                                 the two tables would be as large)             */
    int32_t persistent;       /* 1 = run stretches of events of a species without
                                 reactions in one cooperative launch (default),
                                 -1 = one claim + commit launch per event       */
    int32_t slot_map;         /* home slot of a claim in the hash table:
                                 1 = hashed voxel index (default), 2 = Morton
                                 order, 3 = Morton with permuted low bits      */
    int32_t claim_slots;      /* before populate: hash slots per molecule of
                                 the largest mobile species, rounded up to a
                                 power of two (default 3)                      */
    int32_t run_per_thread;   /* persistent launches: at least this many
                                 molecules per thread (picks the launch shape;
                                 0/-1 = fewest that fit)                       */
    int32_t barrier_timeout_us; /* persistent launches: a block that waits
                                 longer than this at a grid barrier gives up;
                                 the call then fails with PSC_E_TIMEOUT and
                                 the lattice keeps that error (default 10^6)   */
    int32_t barrier_phantom;  /* tests of the time-out path only: arrivals the
                                 grid barrier awaits from blocks that do not
                                 exist, so every persistent launch waits out
                                 barrier_timeout_us (0/-1 = none, default)     */
    int32_t tiles;            /* persistent stretches of a species without
                                 reactions: 1 = owner-computes tile kernel
                                 wherever it applies, -1 = never, 0 = default
                                 (when the species has >= 2^18 molecules on a
                                 lattice of more than 2^22 voxels and,
                                 at its first stretch, the fullest box holds
                                 at most 1.4 x the mean: molecules confined
                                 to part of the lattice take the molecule-
                                 list kernel, which balances itself)           */
    int32_t tile_regions;     /* tile kernel: most boxes (blocks) to cut the
                                 lattice into (0/-1 = one per SM)              */
    int32_t subvolume;        /* before populate: 1 = update rule of the
                                 paper's sub-volume scheme (Sec. 2.5) instead
                                 of the synchronous rule: 2x2x2-voxel
                                 sub-volumes in eight colours taken in an
                                 order drawn per event (draws (a, g, s<<4 | 3),
                                 a = 7..1, Fisher-Yates), sequential in
                                 ascending id within a colour, each molecule
                                 once per event.  Species without reactions
                                 only (else PSC_E_UNSUPPORTED at populate);
                                 periodic extents must be multiples of 4
                                 (PSC_E_DIMS).  -1 = synchronous (default)     */
    int32_t tile_lean;        /* tile kernel variant: 1 = the lean kernel
                                 wherever it applies (default: HCP lattices of
                                 whole 4 x 4 x 2 bricks, boxes at least two
                                 bricks thick, two or more boxes along every
                                 periodic axis), -1 = always the general tile
                                 kernel.  Same results either way              */
} psc_options;

/*
 * Create an empty lattice (Sec. 2.1; FCC: App. B).
 *   ni, nj, nk       extents; a periodic i axis needs ni >= 3, a periodic j
 *                    (k) axis needs an even nj (nk) >= 4 so that the parity
 *                    stencil wraps consistently -- on the FCC lattice a
 *                    periodic k axis needs nk >= 3 and a multiple of 3 (the
 *                    stacking period); ni * nj * nk < 2^31.
 *   voxel_radius_m   r_v in metres (> 0).
 *   boundary_flags   PSC_PERIODIC_* bits, plus PSC_FCC for the FCC lattice:
 *                    the triangular layers stacked ABC, layer k at offset
 *                    (0, 0), (1, 1/sqrt 3) or (0, 2/sqrt 3) r_v for k mod 3 =
 *                    0, 1, 2 (row parity p = (j + [k mod 3 == 1]) & 1).  The
 *                    twelve neighbours are the HCP ones in the layer; below,
 *                    two at i-1+p, i+p on row j+a and one at (i, j+b) with
 *                    (a, b) = (-1, 0) for k mod 3 = 0, else (0, +1); above,
 *                    two on row j+a' and one at (i, j+b') with (a', b') =
 *                    (+1, 0) for k mod 3 = 2, else (0, -1).  Stretches of
 *                    FCC lattices use the molecule-list kernel.
 *   device           CUDA device ordinal.
 *   cuda_stream      cudaStream_t to queue work on, or NULL for a stream the
 *                    library creates and owns.
 * Errors: PSC_E_ARG, PSC_E_DIMS, PSC_E_CUDA.
 */
int psc_lattice_create(psc_lattice **out, int32_t ni, int32_t nj, int32_t nk,
                       double voxel_radius_m, uint32_t boundary_flags,
                       int device, void *cuda_stream);

/* Add a species with diffusion coefficient D (m^2/s, >= 0) and initial count
   (Sec. 2.3).  Before psc_populate only.  Errors: E_ARG, E_ORDER,
   E_UNSUPPORTED (more than PSC_MAX_SPECIES). */
int psc_add_species(psc_lattice *L, double D_m2_s, int64_t initial_count,
                    int32_t *species_out);

/* Register a reaction (Sec. 2.4).  n_reactants = 1: first order, k in 1/s,
   reactant must be mobile; n_reactants = 2: second order, k in m^3/s, two
   different species, one reaction per pair.  0..2 products.  Before populate.
   Errors: E_ARG, E_ORDER, E_UNSUPPORTED (A + A, > 2 products, first order on
   an immobile species, a pair registered twice, more than 8 first-order
   reactions of one species, more than PSC_MAX_REACTIONS). */
int psc_add_reaction(psc_lattice *L, const int32_t *reactants, int32_t n_reactants,
                     const int32_t *products, int32_t n_products, double k,
                     int32_t *reaction_out);

/* Compartments (Sec. 2: a cell is a set of compartments, each a group of
   voxels).  labels: host buffer of V bytes, labels[i + ni (j + nj k)] = the
   compartment of voxel (i, j, k), each below n_compartments (1 ..
   PSC_MAX_COMPARTMENTS); the library copies it, the caller keeps ownership.
   Every species lives in one compartment, 0 unless psc_species_compartment
   says otherwise.  Effects (Sec. 2.3): a hop into a voxel of another
   compartment fails like a hop into an occupied voxel; a collision with a
   registered partner reacts whatever the partner's compartment; products of
   a second-order reaction go to the two reactants' voxels, the first product
   to the partner's and the second to the mover's unless that puts one outside
   its compartment, in which case they trade places (each product takes the id
   of the reactant whose voxel it takes); the second product of a first-order
   reaction goes to a vacant neighbour in its own compartment; placement
   deals each compartment's voxels to its own species.  Before psc_populate;
   calling it again replaces the labels.  Errors: E_ARG (labels NULL, a label
   >= n_compartments, n_compartments out of range, a species already set to a
   compartment >= n_compartments), E_ORDER. */
int psc_set_compartments(psc_lattice *L, const uint8_t *labels, int32_t n_compartments);

/* The compartment species lives in (below the n_compartments of the last
   psc_set_compartments, 0 without one).  Before psc_populate.  Errors: E_ARG,
   E_ORDER. */
int psc_species_compartment(psc_lattice *L, int32_t species, int32_t compartment);

/* Freeze the model, allocate device state and place the molecules uniformly
   at random without replacement (Sec. 3.4 "distributed homogeneously"):
   every voxel gets the key Philox(seed; v, 0, 1, 0) word 0, voxels sorted by
   (key, v) are dealt to the species in index order, ids 0, 1, ... in that
   order (with compartments: each species takes the next voxels of its own
   compartment in that order).  Synchronous.  Returns PSC_W_PCLAMP if some
   p_AB > 1 was clamped.  Errors: E_ARG, E_ORDER (twice), E_FULL (more
   molecules than voxels, in the lattice or in one compartment), E_UNSUPPORTED
   (a reaction whose products cannot all land in their compartments: a
   first-order product that stays must share the reactant's compartment, the
   products of A + B must be one in each reactant's compartment, a single
   one in either), E_NOMEM, E_CUDA. */
int psc_populate(psc_lattice *L, uint64_t seed);

/* Queue every event with time <= t_end (Sec. 2.2); the lattice clock becomes
   max(clock, t_end).  Resumable: run(t1); run(t2) equals run(t2).
   Asynchronous.  Errors: E_ARG (t_end not finite), E_ORDER, E_LIMIT, E_CUDA. */
int psc_run(psc_lattice *L, double t_end);

/* Queue the next n_events events regardless of time (clock = time of the last
   one).  Asynchronous.  Errors as psc_run. */
int psc_run_events(psc_lattice *L, int64_t n_events);

/* Wait for queued work; reports device-side errors (E_CAPACITY, E_TIMEOUT)
   and CUDA errors. */
int psc_synchronize(psc_lattice *L);

/* Molecule counts per species into counts[0 .. n_species-1] (caller-owned,
   n_species >= species added).  Synchronises. */
int psc_counts(psc_lattice *L, int64_t *counts, int32_t n_species);

/* Positions (i, j, k) of the molecules of one species into ijk[3 * a], sorted
   by molecule id, ids into ids[a] if not NULL; *n_out = number of molecules.
   With cap < *n_out nothing is written and E_ARG is returned (call with
   cap = 0 to size the buffers).  Synchronises. */
int psc_coords(psc_lattice *L, int32_t species, int32_t *ijk, uint32_t *ids,
               int64_t cap, int64_t *n_out);

/* Unwrapped positions in the integer basis X = 2I + P, Y = 3J + (K & 1),
   Z = K, where I = i + wraps_i * ni (J, K likewise, wraps counted in 16 bits)
   and P = (J + K) & 1; the centre is (X, Y / sqrt 3, 2 sqrt(2/3) Z) r_v, so
   squared displacements follow exactly (App. C, Eq. 14).  FCC: Y = 3J +
   (K mod 3), P = (J + [K mod 3 == 1]) & 1.  Sorted by id.  Synchronises. */
int psc_unwrapped(psc_lattice *L, int32_t species, int32_t *xyz, uint32_t *ids,
                  int64_t cap, int64_t *n_out);

/* Copy the occupancy grid (ni*nj*nk uint16: 0 vacant, s + 1 species s) into
   occ (caller-owned).  Synchronises. */
int psc_grid(psc_lattice *L, uint16_t *occ);

/* Simulated time (seconds) and number of events queued so far. */
int psc_time(const psc_lattice *L, double *t);
int psc_event_index(const psc_lattice *L, uint32_t *g);

/* Device counters (see psc_stats).  Synchronises. */
int psc_stats_get(psc_lattice *L, psc_stats *s);

/* Sum of the kernel times recorded since the last call (and reset them).
   Synchronises. */
int psc_kernel_times_get(psc_lattice *L, psc_kernel_times *out);

/* Change tunables (psc_options); allowed at any time between calls. */
int psc_set_options(psc_lattice *L, const psc_options *opt);

/*
 * Autotuner: picks the launch options of a lattice by timing real events.
 * It tries, one group after another keeping the best of each, the block
 * shape of the per-event kernels (128 or 256 threads x 4, 8 or 16 blocks per
 * SM), persistent stretches under the tile kernel, under the molecule-list
 * kernel with 0 (fewest that fit), 8 or 16 molecules per thread, or off, and
 * the Morton re-sort period (16 .. 512 events or
 * none; each of these trials starts from freshly sorted lists and spans at
 * least two periods); and, where events take per-event launches, replay
 * from CUDA graphs of 32 or 128 events or none (each trial first runs three
 * runs' worth of events so that its patterns are captured).  Each trial
 * times a window of events with CUDA events on the lattice's stream.  The options change only how the work is laid
 * out on the GPU, never the results (Sec. 2.3's synchronous rule resolves
 * every event from its snapshot and the lowest id), so the trials are real
 * events: the lattice advances by out->events events (at most max_events)
 * and ends bit-identical to a run of that many events without tuning.  The
 * chosen options stay set.  About 3000 events cover every trial; fewer
 * events skip the re-sort periods whose windows no longer fit.
 * Errors: PSC_E_ARG, PSC_E_ORDER (not populated), the lattice's stored error,
 * and those of psc_run_events.
 */
typedef struct {
    int32_t persistent;        /* chosen psc_options values                  */
    int32_t run_per_thread;
    int32_t block_threads;
    int32_t blocks_per_sm;
    int32_t resort_period;     /* -1 = no re-sort                            */
    int32_t tiles;             /* 1 tile kernel, -1 molecule-list kernel     */
    int32_t graph_events;      /* 0 = no graph replay                        */
    int32_t trials;            /* configurations timed                       */
    int64_t events;            /* events the trials ran                      */
    double  us_per_event;      /* of the chosen configuration                */
    double  us_per_event_before; /* of the options in force at the call       */
} psc_tune_result;
int psc_autotune(psc_lattice *L, int64_t max_events, psc_tune_result *out);

/* Hop interval of a species and p_AB of a second-order reaction as the engine
   computes them (Sec. 2.3 Eq. 3, Sec. 2.4.2 Eq. 6; p_AB before clamping). */
double psc_tau(const psc_lattice *L, int32_t species);
double psc_p_ab(const psc_lattice *L, int32_t reaction);

/* Bytes of device memory the lattice holds after psc_populate (or would hold,
   computed from its shape and model, before), including the tile kernel's
   buffers once a stretch has run under it. */
int psc_device_bytes(const psc_lattice *L, int64_t *bytes);

/* Free the lattice and its device memory (waits for its queued work). */
void psc_lattice_destroy(psc_lattice *L);

/* Name of a status code. */
const char *psc_status_string(int status);

/* Install a device allocator for subsequent allocations (NULL, NULL restores
   cudaMalloc / cudaFree).  alloc(bytes, device, stream, ctx) returns a device
   pointer or NULL; release(ptr, device, stream, ctx) frees it.  Process-wide. */
typedef void *(*psc_alloc_fn)(size_t bytes, int device, void *stream, void *ctx);
typedef void (*psc_free_fn)(void *ptr, int device, void *stream, void *ctx);
int psc_set_allocator(psc_alloc_fn alloc, psc_free_fn release, void *ctx);

/*
 * Batches: many lattices (replicas, parameter sweeps) advanced together.
 * Every launch of a batch covers all its members, each running its own next
 * event (its own species and event index), so a batch of small lattices costs
 * about as many launches per event as one lattice.  Results of a member are
 * bit-identical to running it alone (same seed, same model).
 *
 *   psc_batch_create   cuda_stream as for psc_lattice_create.
 *   psc_batch_add      L must be populated, on the batch's device and stream
 *                      (create it with the same cuda_stream), and use one
 *                      claim word per voxel (lattices up to 2^22 voxels by
 *                      default, or psc_options.claim_table = 1); at most 512
 *                      members.  The batch does not own L.
 *   psc_batch_run_events   every member runs n_events more of its events.
 *   psc_batch_run      every member runs its events with time <= t_end.
 * Errors: PSC_E_ARG, PSC_E_ORDER (not populated), PSC_E_UNSUPPORTED (hash
 * claim table, other device or stream), PSC_E_CAPACITY (batch full), PSC_E_CUDA.
 */
typedef struct psc_batch psc_batch;
int  psc_batch_create(psc_batch **out, int device, void *cuda_stream);
int  psc_batch_add(psc_batch *B, psc_lattice *L);
int  psc_batch_remove(psc_batch *B, psc_lattice *L);
int  psc_batch_size(const psc_batch *B, int32_t *n);
int  psc_batch_run_events(psc_batch *B, int64_t n_events);
int  psc_batch_run(psc_batch *B, double t_end);
int64_t psc_batch_launches(const psc_batch *B);
void psc_batch_destroy(psc_batch *B);

/* Batch autotuner: threads per block (128, 256), the most blocks one
   member's event gets in a batched launch (8 .. 256, the rest grid-strided:
   with the threads, the molecules each thread takes), then the members'
   Morton re-sort period (never, or every 64 or 256 of a member's events),
   chosen by timing windows of batched events (CUDA events on the batch's
   stream).  Trial rounds are real events of every member (results are the
   same under any block shape and list order); at most max_rounds batched
   events run.  The chosen options stay set for the batch.  Errors:
   PSC_E_ARG, PSC_E_CUDA. */
typedef struct {
    int32_t threads;
    int32_t blocks_per_member;
    int32_t trials;
    int64_t rounds;            /* batched events the trials ran              */
    double  us_per_round;      /* of the chosen options                      */
    double  us_per_round_before;
    int32_t resort_period;     /* chosen re-sort period of the members (-1 never) */
} psc_batch_tune_result;
int psc_batch_autotune(psc_batch *B, int64_t max_rounds, psc_batch_tune_result *out);

/*
 * Serving: a request loop with continuous batching.  A request describes a
 * whole simulation (lattice, species, reactions, seed, end time); submitted
 * requests wait in FIFO order and are admitted while the device memory they
 * need (psc_device_bytes) fits under max_device_bytes and fewer than
 * max_active run.  psc_server_step admits what fits, advances every admitted
 * simulation by up to n_events of its events in batched launches, and
 * retires the ones that reached their end time (their counts are kept, their
 * memory freed), so requests that arrive while others run join the batch as
 * slots and memory free up.  A result is the same alone and in any mix.
 *   psc_request arrays: D and initial_count have n_species entries; per
 *   reaction r: n_reactants[r] (1|2) reactants at reactants[2r..], n_products[r]
 *   (0..2) products at products[2r..], rate k[r].
 *   psc_server_result: counts at the end time and the seconds from submit to
 *   retirement; PSC_E_ORDER while the request is not finished; the stored
 *   error of a request that failed.
 */
typedef struct {
    int32_t ni, nj, nk;
    uint32_t boundary_flags;
    double voxel_radius_m;
    int32_t n_species;
    const double *D;
    const int64_t *initial_count;
    int32_t n_reactions;
    const int32_t *n_reactants;
    const int32_t *reactants;
    const int32_t *n_products;
    const int32_t *products;
    const double *k;
    uint64_t seed;
    double t_end;
} psc_request;

typedef struct psc_server psc_server;
int  psc_server_create(psc_server **out, int device, void *cuda_stream, int64_t max_device_bytes,
                       int32_t max_active);
int  psc_server_submit(psc_server *S, const psc_request *req, int64_t *ticket);
int  psc_server_step(psc_server *S, int32_t n_events, int32_t *n_active, int32_t *n_waiting);
int  psc_server_result(psc_server *S, int64_t ticket, int64_t *counts, int32_t n_species,
                       double *seconds_to_result);
int  psc_server_memory(const psc_server *S, int64_t *bytes_in_use, int64_t *peak_bytes);
void psc_server_destroy(psc_server *S);

/*
 * Slabs: the lattice split along k into sub-domains, each with a ghost layer on
 * either side refreshed from its neighbours at every event (the paper's
 * sub-domains with ghost voxels, Sec. 2.5), for events of one species without
 * reactions under the synchronous rule.  Slab `index` of `count` owns the
 * layers index * m .. index * m + m - 1, m = nk / count (nk a multiple of
 * count, m >= 2).  An event takes three calls with an exchange with both
 * neighbouring slabs after each of the first two:
 *   psc_slab_claim    directions drawn, vacant targets claimed (lowest id);
 *                     send_claim[0] / [1] hold the claims on the two layers
 *                     at the lower / upper face (a target there can be
 *                     wanted from both sides);
 *   psc_slab_commit   recv_claim[0] / [1] (the neighbours' send_claim[1] /
 *                     [0]) are merged, winners move; send_commit[side] holds
 *                     the molecules that entered that neighbour's layers and
 *                     this slab's boundary layer on that side;
 *   psc_slab_apply    recv_commit[0] / [1] (the neighbours' send_commit[1] /
 *                     [0]) refresh the ghost layers and add the arrivals.
 * Side 0 is the lower neighbour (index - 1), side 1 the upper one (index + 1);
 * along a periodic k axis slab 0 and slab count - 1 are neighbours (with one
 * slab, the slab is its own neighbour), along a reflective one the outer
 * sides exchange nothing.  Results are bit-identical to psc_run_events on the
 * whole lattice (same seed and event indices).
 *
 *   psc_slab_create   from a populated lattice L: its only mobile species is
 *                     `species`, which has no reactions (others immobile,
 *                     else PSC_E_UNSUPPORTED; HCP only); copies the slab's
 *                     share of L's molecules and occupancy and L's event
 *                     index; device and cuda_stream (NULL: a stream the slab
 *                     owns) for the slab's state.  L stays as it was.
 *   psc_slab_buffers_get / _set   the eight exchange buffers (device memory
 *                     of claim_bytes or commit_bytes each) the slab allocated,
 *                     or ones the caller provides instead (e.g. buffers a
 *                     collective library sends and receives); the caller
 *                     keeps ownership of buffers it sets.
 *   psc_slabs_run_events   n_events events of slabs[0 .. count - 1] (all of
 *                     one split, index order) in this process, exchanging
 *                     by device copies (peer copies across devices).
 *   psc_slab_coords   the slab's molecules: global (i, j, k) into ijk[3 a],
 *                     ids, unwrapped positions as psc_unwrapped (xyz may be
 *                     NULL), in list order; *n_out = count (cap = 0 sizes).
 *   psc_slab_synchronize  waits; reports PSC_E_CAPACITY if a list or a
 *                     message overflowed.
 * Errors: PSC_E_ARG, PSC_E_ORDER (L not populated), PSC_E_DIMS,
 * PSC_E_UNSUPPORTED, PSC_E_NOMEM, PSC_E_CAPACITY, PSC_E_LIMIT, PSC_E_CUDA.
 */
typedef struct psc_slab psc_slab;
typedef struct {
    void *send_claim[2], *recv_claim[2], *send_commit[2], *recv_commit[2];
} psc_slab_buffers;
int  psc_slab_create(psc_slab **out, psc_lattice *L, int32_t species, int32_t index, int32_t count,
                     int device, void *cuda_stream);
int  psc_slab_buffers_get(const psc_slab *S, psc_slab_buffers *b, int64_t *claim_bytes,
                          int64_t *commit_bytes);
int  psc_slab_buffers_set(psc_slab *S, const psc_slab_buffers *b);
int  psc_slab_claim(psc_slab *S);
int  psc_slab_commit(psc_slab *S);
int  psc_slab_apply(psc_slab *S);
int  psc_slabs_run_events(psc_slab **slabs, int32_t count, int64_t n_events);
int  psc_slab_synchronize(psc_slab *S);
int  psc_slab_coords(psc_slab *S, int32_t *ijk, uint32_t *ids, int32_t *xyz, int64_t cap, int64_t *n_out);
int  psc_slab_event_index(const psc_slab *S, uint32_t *g);
void psc_slab_destroy(psc_slab *S);

/*
 * psc_hop_events_static -- n_events diffusion events of one species that has
 * no reactions, on molecule buffers the caller owns, without allocating any
 * memory.  (The paper has no counterpart: this is a deployment variant of
 * the claim/commit kernels of psc_run_events.)
 *
 * For callers that cannot allocate device memory when they step molecules --
 * a framework that owns all device memory through its own pool, code running
 * under an allocator lock, or code that must not trigger the synchronisation
 * cudaMalloc/cudaFree may cause.  The claim words, the vacancy mirror and the
 * counters live in fixed-size device arrays inside the library, which every
 * GPU that loads the library holds until the process exits (about 12 MiB).
 *
 *   ni, nj, nk, boundary_flags   lattice as for psc_lattice_create; at most
 *                    2^21 voxels (e.g. 128^3) and a vacancy mirror of at most
 *                    2^20 words, else PSC_E_CAPACITY.
 *   seed, species    Philox key and species index of the draws; with
 *                    first_event the event index of the first event, so the
 *                    results equal psc_run_events on a lattice holding the
 *                    same molecules with the same seed (bit for bit).
 *   vox              device, n entries, in/out: voxel index of each molecule;
 *                    each in [0, ni*nj*nk) and no two equal.
 *   ids              device, n entries, in: molecule ids, distinct and below
 *                    0xFFFFFFFF (that value marks an unclaimed voxel).
 *   img              device, n entries, in/out: packed 16-bit wrap counters
 *                    (i bits 0-15, j 16-31, k 32-47); zeros if unused.
 *   n                molecules (the only occupied voxels of the lattice).
 *   stream           cudaStream_t (NULL = default stream).
 * The call queues its work on the stream, waits for it (the stream is
 * synchronised) and returns the status the device raised.  Every call first
 * clears ni*nj*nk claim words and the vacancy mirror (about 4.5 bytes per
 * voxel) and rebuilds the mirror from vox, so batch many events into one
 * call.  The molecules are checked on the device while the mirror is built:
 * an entry whose voxel is out of range or already taken, or whose id is
 * 0xFFFFFFFF, is skipped, no event runs, the caller's buffers are left as
 * they were and the call returns PSC_E_ARG.  Distinct ids are not checked:
 * with two equal ids the results are undefined (every access stays in
 * bounds).  The first call on each device looks up the addresses of the
 * internal arrays (cudaGetSymbolAddress) with that device current; make it
 * before any stream capture.  All calls on a device share the arrays, which
 * keep the last call's contents: calls that may overlap on the GPU
 * (different streams, or host threads) race and must be serialised by the
 * caller.
 * Errors: PSC_E_ARG (null buffer, bad species or flags, bad molecules as
 * above), PSC_E_DIMS, PSC_E_FULL, PSC_E_LIMIT, PSC_E_CAPACITY (lattice above
 * the limit), PSC_E_CUDA.
 */
int psc_hop_events_static(int32_t ni, int32_t nj, int32_t nk, uint32_t boundary_flags,
                          uint64_t seed, int32_t species, uint32_t first_event, int32_t n_events,
                          int32_t *vox, const uint32_t *ids, uint64_t *img, int32_t n, void *stream);

#ifdef __cplusplus
}
#endif
#endif
