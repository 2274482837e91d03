/*
 * psco.h -- plain, slow CPU oracle for the pSpatiocyte voxel hop step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this code; only the test-suite, the smoke check and the timed CPU
 * baseline of the benchmark may.  It shares no source with the CUDA path:
 * geometry, random numbers, thresholds, the scheduler and both update rules
 * are written here a second time, straight from the paper's definitions.
 *
 * Paper: Miyauchi, Iwamoto, Arjunan, Takahashi, "pSpatiocyte: A Parallel
 * Stochastic Method for Particle Reaction-Diffusion Systems" (arXiv 1605.03726).
 *   Sec. 2.1      HCP lattice in twisted Cartesian coordinates (12 neighbours,
 *                 stencil chosen by the parity of the j and k layers); App. B
 *                 (figures only) the FCC lattice in the same coordinates, ABC
 *                 stacking (layer offsets chosen by k mod 3).
 *   Sec. 2.2      event scheduler: per-species diffusion events in time order.
 *   Sec. 2        compartments: groups of voxels; every species lives in one.
 *   Sec. 2.3      diffusion: hop interval tau_d = 2 r_v^2 / (3 D); a molecule
 *                 moves to a randomly chosen neighbour only if it is vacant
 *                 and in the molecule's compartment.
 *   Sec. 2.4.1    first-order reactions (modified Gillespie direct method).
 *   Sec. 2.4.2    second-order reactions, discrete Collins-Kimball acceptance
 *                 p_AB = k / (6 sqrt(2) (D_A + D_B) r_v) on collision.
 *   App. C        Einstein-Smoluchowski relation lambda^2 = 6 D t.
 *
 * Two update rules are provided:
 *   PSCO_RULE_SYNC        every molecule of the due species decides against the
 *                         grid as it was when the event began; a contested
 *                         target goes to the lowest molecule id.
 *   PSCO_RULE_SEQ_ID      the paper's one-by-one update (Sec. 2.3) in ascending
 *                         id order, each molecule seeing the current grid.
 *   PSCO_RULE_SEQ_RANDOM  the same, in a fresh random order every event.
 *   PSCO_RULE_SUBVOL      the paper's sub-volume scheme (Sec. 2.5) on the
 *                         lattice: 2 x 2 x 2-voxel sub-volumes coloured by the
 *                         parities of their indices; each event takes the eight
 *                         colours in an order drawn for it, and within a colour
 *                         the molecules standing in sub-volumes of that colour,
 *                         not yet processed in the event, one by one in
 *                         ascending id, each seeing the current grid.
 * All use the same per-molecule draws.
 */
#ifndef PSCO_H
#define PSCO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PSCO_OK              0
#define PSCO_E_ARG          -1
#define PSCO_E_DIMS         -2
#define PSCO_E_ORDER        -3
#define PSCO_E_FULL         -4
#define PSCO_E_UNSUPPORTED  -5
#define PSCO_E_NOMEM        -6
#define PSCO_E_LIMIT        -9
#define PSCO_W_PCLAMP        1

#define PSCO_RULE_SYNC        0
#define PSCO_RULE_SEQ_ID      1
#define PSCO_RULE_SEQ_RANDOM  2
#define PSCO_RULE_SUBVOL      3   /* periodic axes need extents that are multiples of 4 */

#define PSCO_MAX_SPECIES    64
#define PSCO_MAX_REACTIONS 256
#define PSCO_MAX_COMPARTMENTS 16

/* boundary flag bits: set = periodic, clear = reflective wall */
#define PSCO_PERIODIC_I 1u
#define PSCO_PERIODIC_J 2u
#define PSCO_PERIODIC_K 4u
/* lattice flag bit: set = FCC (ABC stacking), clear = HCP (ABAB) */
#define PSCO_FCC        8u

typedef struct psco_lattice psco_lattice;

/* counters accumulated over all events */
typedef struct {
    uint64_t attempts;      /* molecules processed, whatever the outcome       */
    uint64_t hops;          /* successful moves into a vacant voxel            */
    uint64_t collisions;    /* targets holding a registered reaction partner   */
    uint64_t accepted;      /* collisions whose acceptance draw passed         */
    uint64_t reactions2;    /* second-order reactions carried out              */
    uint64_t fires;         /* first-order firings (draw passed)               */
    uint64_t reactions1;    /* first-order reactions carried out               */
    uint64_t births;        /* molecules given a fresh id                      */
    uint64_t events;        /* species events processed                        */
    uint64_t dir_count[12]; /* chosen hop direction histogram                  */
} psco_stats;

int  psco_lattice_create(psco_lattice **out, int32_t ni, int32_t nj, int32_t nk,
                         double voxel_radius_m, uint32_t boundary_flags, int32_t rule);
int  psco_add_species(psco_lattice *L, double D_m2_s, int64_t initial_count,
                      int32_t *species_out);
int  psco_add_reaction(psco_lattice *L, const int32_t *reactants, int32_t n_reactants,
                       const int32_t *products, int32_t n_products, double k,
                       int32_t *reaction_out);
/* compartments (Sec. 2; before populate): labels[v], v = i + ni (j + nj k),
   in [0, n); a species lives in compartment 0 unless set.  A hop into a
   voxel of another compartment fails (Sec. 2.3); collisions with partners
   react across compartments; placement fills each compartment on its own. */
int  psco_set_compartments(psco_lattice *L, const uint8_t *labels, int32_t n_compartments);
int  psco_species_compartment(psco_lattice *L, int32_t species, int32_t compartment);
int  psco_populate(psco_lattice *L, uint64_t seed);
int  psco_run(psco_lattice *L, double t_end);
int  psco_run_events(psco_lattice *L, int64_t n_events);
int  psco_counts(const psco_lattice *L, int64_t *counts, int32_t n_species);
int  psco_coords(const psco_lattice *L, int32_t species, int32_t *ijk, uint32_t *ids,
                 int64_t cap, int64_t *n_out);
int  psco_unwrapped(const psco_lattice *L, int32_t species, int32_t *xyz,
                    uint32_t *ids, int64_t cap, int64_t *n_out);
int  psco_grid(const psco_lattice *L, uint16_t *occ);
int  psco_time(const psco_lattice *L, double *t);
int  psco_event_index(const psco_lattice *L, uint32_t *g);
int  psco_stats_get(const psco_lattice *L, psco_stats *s);
int  psco_check(const psco_lattice *L);     /* 0 if grid, molecules and compartments agree */
/* test helper: after populate, put one molecule of `species` on vacant voxel v;
   it takes the next fresh id */
int  psco_place(psco_lattice *L, int32_t species, int32_t v, uint32_t *id_out);
void psco_lattice_destroy(psco_lattice *L);

/* derived constants, exposed for the pins */
double   psco_tau(const psco_lattice *L, int32_t species);        /* Sec. 2.3     */
double   psco_p_ab(const psco_lattice *L, int32_t reaction);      /* Sec. 2.4.2   */
uint64_t psco_threshold(double p);          /* floor(min(p,1) * 2^32)             */

/* primitives, exposed for the pins */
void psco_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int  psco_neighbor(const psco_lattice *L, int32_t i, int32_t j, int32_t k, int32_t d,
                   int32_t out_ijk[3], int32_t wrap[3]);   /* 1 = inside, 0 = wall */
void psco_center(int32_t i, int32_t j, int32_t k, double xyz[3]);  /* units of r_v */
void psco_center_fcc(int32_t i, int32_t j, int32_t k, double xyz[3]);   /* FCC lattice */

#ifdef __cplusplus
}
#endif
#endif
