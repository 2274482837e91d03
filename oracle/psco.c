/*
 * psco.c -- plain, slow CPU oracle for the pSpatiocyte voxel hop step.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
 * timed CPU baseline, never by the product library.  Written for clarity: one
 * molecule at a time, library qsort for every ordering step, no blocking or
 * fusion.  Every function names the passage of the paper it follows.
 *
 * Parity status of each part (pins live in tests/test_oracle_*.py):
 *   philox        pinned to cuRAND's host Philox4x32-10 generator.
 *   geometry      pinned by brute-force nearest-neighbour search on the
 *                 HCP centres (Sec. 2.1, Fig. 3/4), exact 2 r_v spacing,
 *                 symmetry, ABAB stacking.
 *   diffusion     pinned by MSD = 6 D t (Eq. 2 / App. C) and by exact
 *                 enumeration of one-event transition probabilities.
 *   first order   pinned by A(t) = A0 exp(-k t) (Sec. 3.2.1).
 *   second order  pinned by the accepted fraction of collisions = p_AB
 *                 (Sec. 2.4.2) and by mass action at low p.
 *   sync rule     pinned by exact enumeration on tiny lattices.
 */
#include "psco.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), replacing the paper's   */
/* Mersenne Twister (Sec. 2.5) by a counter-based generator so that a draw is */
/* a pure function of (seed, event, molecule).                                */
/* ------------------------------------------------------------------------ */
void psco_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;      /* golden ratio          */
            k1 += 0xBB67AE85u;      /* sqrt(3) - 1           */
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* counter word 2 carries the species and a domain tag */
#define TAG_EVENT    0u
#define TAG_POPULATE 1u
#define TAG_ORDER    2u
#define TAG_SUBVOL   3u

static void draw(const psco_lattice *L, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t u[4]);

/* ------------------------------------------------------------------------ */
/* state                                                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t  v;          /* voxel index i + ni*(j + nj*k)          */
    uint32_t id;
    int16_t  img[3];     /* periodic wrap counters (16-bit, wrapping) */
    int16_t  species;    /* -1 once the molecule is gone            */
} omol;

typedef struct {
    double   D;
    int64_t  n0;
    double   tau;        /* hop interval, Sec. 2.3                   */
    uint64_t done;       /* diffusion events processed               */
    int32_t  n_fo;       /* first-order reactions of this species    */
    int32_t  fo[PSCO_MAX_REACTIONS];
    uint64_t T_fire;     /* per-event firing threshold               */
    uint64_t cum[PSCO_MAX_REACTIONS];  /* choice thresholds           */
    int64_t *list;       /* indices into mol[] (rebuilt when dirty)  */
    int64_t  nlist;
    int      dirty;
    int32_t  comp;       /* compartment the species lives in (Sec. 2) */
} ospec;

typedef struct {
    int32_t nr, np;
    int32_t r[2], p[2];
    double  k;
    double  prob;        /* p_AB for second order                    */
    uint64_t T;          /* acceptance threshold                     */
} orx;

struct psco_lattice {
    int32_t  ni, nj, nk;
    int64_t  V;
    double   rv;
    uint32_t bflags;
    int32_t  rule;
    int32_t  nsp;
    ospec    sp[PSCO_MAX_SPECIES];
    int32_t  nrx;
    orx      rx[PSCO_MAX_REACTIONS];
    int16_t  pair[PSCO_MAX_SPECIES][PSCO_MAX_SPECIES];
    uint16_t *occ;       /* 0 vacant, s+1 species s                  */
    uint8_t  *comp;      /* compartment of every voxel, NULL = all 0 */
    int32_t  ncomp;
    int64_t  *who;       /* voxel -> index into mol[], -1 if vacant  */
    omol     *mol;
    int64_t  nmol, capmol;
    uint64_t seed;
    int      populated;
    uint32_t g;          /* global event index                       */
    uint32_t next_id;
    double   clock;
    psco_stats st;
};

static void draw(const psco_lattice *L, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t u[4])
{
    uint32_t ctr[4] = { c0, c1, c2, 0u };
    uint32_t key[2] = { (uint32_t)L->seed, (uint32_t)(L->seed >> 32) };
    psco_philox4x32_10(ctr, key, u);
}

/* ------------------------------------------------------------------------ */
/* geometry: Sec. 2.1 twisted Cartesian coordinates on the HCP lattice.       */
/* i is the straight axis, j and k the zigzag axes; p = (j + k) & 1 selects   */
/* the stencil.  Centres (units of r_v): x = 2i + p, y = sqrt(3) j + (k&1)/   */
/* sqrt(3), z = 2 sqrt(2/3) k -- layers k and k+2 coincide (ABAB, HCP).       */
/* ------------------------------------------------------------------------ */
void psco_center(int32_t i, int32_t j, int32_t k, double xyz[3])
{
    int p = (j + k) & 1;
    xyz[0] = 2.0 * i + p;
    xyz[1] = sqrt(3.0) * j + (double)(k & 1) / sqrt(3.0);
    xyz[2] = 2.0 * sqrt(2.0 / 3.0) * k;
}

/* FCC (App. B, figures only; derived here): the same triangular layers in
   ABC stacking.  Layer k sits at (0, 0), (1, 1/sqrt(3)) or (0, 2/sqrt(3))
   for k mod 3 = 0, 1, 2, so with c = k mod 3 and row parity
   p = (j + [c == 1]) & 1 the centre is x = 2i + p, y = sqrt(3) j + c/sqrt(3),
   z = 2 sqrt(2/3) k; layers k and k+3 coincide. */
void psco_center_fcc(int32_t i, int32_t j, int32_t k, double xyz[3])
{
    int c = ((k % 3) + 3) % 3;
    int p = (j + (c == 1)) & 1;
    xyz[0] = 2.0 * i + p;
    xyz[1] = sqrt(3.0) * j + (double)c / sqrt(3.0);
    xyz[2] = 2.0 * sqrt(2.0 / 3.0) * k;
}

/* FCC neighbour offsets, d = 0..11 in the HCP order: the six in the layer as
   for HCP; below, two at (i-1+p, i+p) on row j + a and one at (i, j + b) with
   (a, b) = (-1, 0) for c = 0 and (0, +1) otherwise; above, two on row j + a'
   and one at (i, j + b') with (a', b') = (+1, 0) for c = 2 and (0, -1)
   otherwise. */
static void raw_neighbor_fcc(int32_t i, int32_t j, int32_t k, int32_t d, int32_t o[3])
{
    int c = ((k % 3) + 3) % 3;
    int p = (j + (c == 1)) & 1;
    int ab = c == 0 ? -1 : 0, bb = c == 0 ? 0 : 1;
    int aa = c == 2 ? 1 : 0, ba = c == 2 ? 0 : -1;
    switch (d) {
    case 0:  o[0] = i + 1;     o[1] = j;      o[2] = k;     break;
    case 1:  o[0] = i - 1;     o[1] = j;      o[2] = k;     break;
    case 2:  o[0] = i - 1 + p; o[1] = j - 1;  o[2] = k;     break;
    case 3:  o[0] = i + p;     o[1] = j - 1;  o[2] = k;     break;
    case 4:  o[0] = i - 1 + p; o[1] = j + 1;  o[2] = k;     break;
    case 5:  o[0] = i + p;     o[1] = j + 1;  o[2] = k;     break;
    case 6:  o[0] = i - 1 + p; o[1] = j + ab; o[2] = k - 1; break;
    case 7:  o[0] = i + p;     o[1] = j + ab; o[2] = k - 1; break;
    case 8:  o[0] = i;         o[1] = j + bb; o[2] = k - 1; break;
    case 9:  o[0] = i - 1 + p; o[1] = j + aa; o[2] = k + 1; break;
    case 10: o[0] = i + p;     o[1] = j + aa; o[2] = k + 1; break;
    default: o[0] = i;         o[1] = j + ba; o[2] = k + 1; break;
    }
}

/* the 12 neighbour offsets; d = 0..11 in this fixed order */
static void raw_neighbor(int32_t i, int32_t j, int32_t k, int32_t d, int32_t o[3])
{
    int p = (j + k) & 1;
    int dj = (k & 1) ? 1 : -1;            /* in-plane shift of the apex neighbours */
    switch (d) {
    case 0:  o[0] = i + 1;     o[1] = j;      o[2] = k;     break;
    case 1:  o[0] = i - 1;     o[1] = j;      o[2] = k;     break;
    case 2:  o[0] = i - 1 + p; o[1] = j - 1;  o[2] = k;     break;
    case 3:  o[0] = i + p;     o[1] = j - 1;  o[2] = k;     break;
    case 4:  o[0] = i - 1 + p; o[1] = j + 1;  o[2] = k;     break;
    case 5:  o[0] = i + p;     o[1] = j + 1;  o[2] = k;     break;
    case 6:  o[0] = i - 1 + p; o[1] = j;      o[2] = k - 1; break;
    case 7:  o[0] = i + p;     o[1] = j;      o[2] = k - 1; break;
    case 8:  o[0] = i;         o[1] = j + dj; o[2] = k - 1; break;
    case 9:  o[0] = i - 1 + p; o[1] = j;      o[2] = k + 1; break;
    case 10: o[0] = i + p;     o[1] = j;      o[2] = k + 1; break;
    default: o[0] = i;         o[1] = j + dj; o[2] = k + 1; break;
    }
}

int psco_neighbor(const psco_lattice *L, int32_t i, int32_t j, int32_t k, int32_t d,
                  int32_t out[3], int32_t wrap[3])
{
    int32_t o[3];
    int32_t n[3] = { L->ni, L->nj, L->nk };
    if (L->bflags & PSCO_FCC) raw_neighbor_fcc(i, j, k, d, o);
    else raw_neighbor(i, j, k, d, o);
    for (int a = 0; a < 3; ++a) {
        wrap[a] = 0;
        if (o[a] < 0 || o[a] >= n[a]) {
            if (!(L->bflags & (1u << a)))
                return 0;                   /* reflective wall: the hop fails (Sec. 2.3) */
            if (o[a] < 0) { o[a] += n[a]; wrap[a] = -1; }
            else          { o[a] -= n[a]; wrap[a] = +1; }
        }
        out[a] = o[a];
    }
    return 1;
}

static void decode(const psco_lattice *L, int64_t v, int32_t ijk[3])
{
    ijk[0] = (int32_t)(v % L->ni);
    ijk[1] = (int32_t)((v / L->ni) % L->nj);
    ijk[2] = (int32_t)(v / ((int64_t)L->ni * L->nj));
}

/* compartment of voxel v (Sec. 2: a cell is a set of compartments, each a
   group of voxels) */
static int32_t vcomp(const psco_lattice *L, int64_t v)
{
    return L->comp ? (int32_t)L->comp[v] : 0;
}

static int64_t encode(const psco_lattice *L, const int32_t ijk[3])
{
    return (int64_t)ijk[0] + (int64_t)L->ni * ((int64_t)ijk[1] + (int64_t)L->nj * ijk[2]);
}

/* ------------------------------------------------------------------------ */
/* constants                                                                  */
/* ------------------------------------------------------------------------ */
uint64_t psco_threshold(double p)
{
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return (uint64_t)1 << 32;
    return (uint64_t)floor(p * 4294967296.0);
}

/* Sec. 2.3: tau_d = 2 r_v^2 / (3 D) */
static double hop_interval(double rv, double D)
{
    return (2.0 * rv * rv) / (3.0 * D);
}

/* Sec. 2.4.2: p_AB = k_AB / (6 sqrt(2) (D_A + D_B) r_v) */
static double collision_probability(double k, double DA, double DB, double rv)
{
    return k / (6.0 * sqrt(2.0) * (DA + DB) * rv);
}

double psco_tau(const psco_lattice *L, int32_t s)
{
    if (!L || s < 0 || s >= L->nsp || !(L->sp[s].D > 0.0)) return 0.0;
    return hop_interval(L->rv, L->sp[s].D);
}

double psco_p_ab(const psco_lattice *L, int32_t r)
{
    if (!L || r < 0 || r >= L->nrx || L->rx[r].nr != 2) return 0.0;
    return collision_probability(L->rx[r].k, L->sp[L->rx[r].r[0]].D,
                                 L->sp[L->rx[r].r[1]].D, L->rv);
}

/* ------------------------------------------------------------------------ */
/* construction                                                               */
/* ------------------------------------------------------------------------ */
int psco_lattice_create(psco_lattice **out, int32_t ni, int32_t nj, int32_t nk,
                        double rv, uint32_t bflags, int32_t rule)
{
    if (!out) return PSCO_E_ARG;
    *out = NULL;
    if (!(rv > 0.0) || !isfinite(rv) || bflags > 15u) return PSCO_E_ARG;
    if (rule < PSCO_RULE_SYNC || rule > PSCO_RULE_SUBVOL) return PSCO_E_ARG;
    if (ni < 1 || nj < 1 || nk < 1) return PSCO_E_DIMS;
    int64_t V = (int64_t)ni * nj * nk;
    if (V >= ((int64_t)1 << 31)) return PSCO_E_DIMS;
    /* periodic wrap keeps the parity stencil consistent only for even j and k
       extents (Sec. 2.1), and 12 distinct neighbours need at least 3 / 4 / 4 */
    if ((bflags & PSCO_PERIODIC_I) && ni < 3) return PSCO_E_DIMS;
    if ((bflags & PSCO_PERIODIC_J) && (nj < 4 || (nj & 1))) return PSCO_E_DIMS;
    if (!(bflags & PSCO_FCC) && (bflags & PSCO_PERIODIC_K) && (nk < 4 || (nk & 1))) return PSCO_E_DIMS;
    if ((bflags & PSCO_FCC) && (bflags & PSCO_PERIODIC_K) && (nk < 3 || nk % 3)) return PSCO_E_DIMS;
    /* sub-volume colours must alternate across a periodic wrap */
    if (rule == PSCO_RULE_SUBVOL && (((bflags & PSCO_PERIODIC_I) && ni % 4) || ((bflags & PSCO_PERIODIC_J) && nj % 4) ||
                                     ((bflags & PSCO_PERIODIC_K) && nk % 4)))
        return PSCO_E_DIMS;
    psco_lattice *L = (psco_lattice *)calloc(1, sizeof(psco_lattice));
    if (!L) return PSCO_E_NOMEM;
    L->ni = ni; L->nj = nj; L->nk = nk; L->V = V;
    L->rv = rv; L->bflags = bflags; L->rule = rule;
    L->ncomp = 1;
    for (int a = 0; a < PSCO_MAX_SPECIES; ++a)
        for (int b = 0; b < PSCO_MAX_SPECIES; ++b)
            L->pair[a][b] = -1;
    *out = L;
    return PSCO_OK;
}

int psco_add_species(psco_lattice *L, double D, int64_t n0, int32_t *species_out)
{
    if (!L) return PSCO_E_ARG;
    if (L->populated) return PSCO_E_ORDER;
    if (!(D >= 0.0) || !isfinite(D) || n0 < 0) return PSCO_E_ARG;
    if (L->nsp >= PSCO_MAX_SPECIES) return PSCO_E_UNSUPPORTED;
    ospec *S = &L->sp[L->nsp];
    memset(S, 0, sizeof(*S));
    S->D = D;
    S->n0 = n0;
    S->tau = D > 0.0 ? hop_interval(L->rv, D) : 0.0;
    S->dirty = 1;
    if (species_out) *species_out = L->nsp;
    L->nsp++;
    return PSCO_OK;
}

int psco_add_reaction(psco_lattice *L, const int32_t *re, int32_t nr,
                      const int32_t *pr, int32_t np, double k, int32_t *rx_out)
{
    if (!L) return PSCO_E_ARG;
    if (L->populated) return PSCO_E_ORDER;
    if (nr < 1 || nr > 2 || np < 0 || !re || (np > 0 && !pr)) return PSCO_E_ARG;
    if (!(k >= 0.0) || !isfinite(k)) return PSCO_E_ARG;
    if (np > 2) return PSCO_E_UNSUPPORTED;
    for (int a = 0; a < nr; ++a)
        if (re[a] < 0 || re[a] >= L->nsp) return PSCO_E_ARG;
    for (int a = 0; a < np; ++a)
        if (pr[a] < 0 || pr[a] >= L->nsp) return PSCO_E_ARG;
    if (L->nrx >= PSCO_MAX_REACTIONS) return PSCO_E_UNSUPPORTED;
    if (nr == 2) {
        if (re[0] == re[1]) return PSCO_E_UNSUPPORTED;             /* A + A     */
        if (!(L->sp[re[0]].D + L->sp[re[1]].D > 0.0)) return PSCO_E_UNSUPPORTED;
        if (L->pair[re[0]][re[1]] >= 0) return PSCO_E_UNSUPPORTED; /* one per pair */
    } else {
        if (!(L->sp[re[0]].D > 0.0)) return PSCO_E_UNSUPPORTED;    /* no events */
    }
    orx *R = &L->rx[L->nrx];
    memset(R, 0, sizeof(*R));
    R->nr = nr; R->np = np; R->k = k;
    for (int a = 0; a < nr; ++a) R->r[a] = re[a];
    for (int a = 0; a < np; ++a) R->p[a] = pr[a];
    if (nr == 2) {
        L->pair[re[0]][re[1]] = (int16_t)L->nrx;
        L->pair[re[1]][re[0]] = (int16_t)L->nrx;
    } else {
        ospec *S = &L->sp[re[0]];
        S->fo[S->n_fo++] = L->nrx;
    }
    if (rx_out) *rx_out = L->nrx;
    L->nrx++;
    return PSCO_OK;
}

/* compartments (Sec. 2): labels[v] for v = i + ni (j + nj k), each below n */
int psco_set_compartments(psco_lattice *L, const uint8_t *labels, int32_t n)
{
    if (!L || !labels) return PSCO_E_ARG;
    if (L->populated) return PSCO_E_ORDER;
    if (n < 1 || n > PSCO_MAX_COMPARTMENTS) return PSCO_E_ARG;
    for (int64_t v = 0; v < L->V; ++v)
        if (labels[v] >= n) return PSCO_E_ARG;
    for (int s = 0; s < L->nsp; ++s)
        if (L->sp[s].comp >= n) return PSCO_E_ARG;
    uint8_t *c = (uint8_t *)malloc((size_t)L->V);
    if (!c) return PSCO_E_NOMEM;
    memcpy(c, labels, (size_t)L->V);
    free(L->comp);
    L->comp = c;
    L->ncomp = n;
    return PSCO_OK;
}

int psco_species_compartment(psco_lattice *L, int32_t s, int32_t c)
{
    if (!L || s < 0 || s >= L->nsp) return PSCO_E_ARG;
    if (L->populated) return PSCO_E_ORDER;
    if (c < 0 || c >= L->ncomp) return PSCO_E_ARG;
    L->sp[s].comp = c;
    return PSCO_OK;
}

/* Reactions must leave every product in its own compartment, given where the
   products go: a first-order product that stays keeps the reactant's voxel;
   a second-order reaction puts its products on the two reactants' voxels. */
static int reactions_fit_compartments(const psco_lattice *L)
{
    for (int r = 0; r < L->nrx; ++r) {
        const orx *R = &L->rx[r];
        int32_t ca = L->sp[R->r[0]].comp;
        if (R->nr == 1) {
            if (R->np >= 1 && L->sp[R->p[0]].comp != ca) return 0;
            continue;
        }
        int32_t cb = L->sp[R->r[1]].comp;
        if (R->np == 1) {
            int32_t c0 = L->sp[R->p[0]].comp;
            if (c0 != ca && c0 != cb) return 0;
        } else if (R->np == 2) {
            int32_t c0 = L->sp[R->p[0]].comp, c1 = L->sp[R->p[1]].comp;
            if (!((c0 == ca && c1 == cb) || (c0 == cb && c1 == ca))) return 0;
        }
    }
    return 1;
}

void psco_lattice_destroy(psco_lattice *L)
{
    if (!L) return;
    for (int s = 0; s < L->nsp; ++s) free(L->sp[s].list);
    free(L->occ); free(L->who); free(L->mol); free(L->comp);
    free(L);
}

/* ------------------------------------------------------------------------ */
/* molecules                                                                  */
/* ------------------------------------------------------------------------ */
static int64_t mol_new(psco_lattice *L)
{
    if (L->nmol == L->capmol) {
        int64_t cap = L->capmol ? 2 * L->capmol : 1024;
        omol *m = (omol *)realloc(L->mol, (size_t)cap * sizeof(omol));
        if (!m) return -1;
        L->mol = m;
        L->capmol = cap;
    }
    return L->nmol++;
}

static void set_species(psco_lattice *L, int64_t m, int32_t s)
{
    int32_t old = L->mol[m].species;
    if (old >= 0) L->sp[old].dirty = 1;
    if (s >= 0) L->sp[s].dirty = 1;
    L->mol[m].species = (int16_t)s;
}

/* list of molecules of species s, ascending id */
static const psco_lattice *g_sort_ctx;
static int cmp_index_by_id(const void *a, const void *b)
{
    uint32_t x = g_sort_ctx->mol[*(const int64_t *)a].id;
    uint32_t y = g_sort_ctx->mol[*(const int64_t *)b].id;
    return (x > y) - (x < y);
}

static int rebuild_list(psco_lattice *L, int32_t s)
{
    ospec *S = &L->sp[s];
    if (!S->dirty) return PSCO_OK;
    int64_t n = 0;
    for (int64_t m = 0; m < L->nmol; ++m)
        if (L->mol[m].species == s) ++n;
    int64_t *lst = (int64_t *)realloc(S->list, (size_t)(n ? n : 1) * sizeof(int64_t));
    if (!lst) return PSCO_E_NOMEM;
    S->list = lst;
    n = 0;
    for (int64_t m = 0; m < L->nmol; ++m)
        if (L->mol[m].species == s) lst[n++] = m;
    g_sort_ctx = L;
    qsort(lst, (size_t)n, sizeof(int64_t), cmp_index_by_id);
    S->nlist = n;
    S->dirty = 0;
    return PSCO_OK;
}

/* ------------------------------------------------------------------------ */
/* populate: uniform placement without replacement ("distributed            */
/* homogeneously", Sec. 3.4).  Every voxel gets a Philox key; voxels sorted by */
/* (key, voxel) are dealt out to the species in index order; ids 0, 1, ...   */
/* follow that order.                                                         */
/* ------------------------------------------------------------------------ */
static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static int freeze_constants(psco_lattice *L)
{
    int clamped = 0;
    for (int r = 0; r < L->nrx; ++r) {
        orx *R = &L->rx[r];
        if (R->nr == 2) {
            R->prob = collision_probability(R->k, L->sp[R->r[0]].D, L->sp[R->r[1]].D, L->rv);
            if (R->prob > 1.0) clamped = 1;       /* p_AB > 1 is clamped to 1 */
            R->T = psco_threshold(R->prob);
        }
    }
    for (int s = 0; s < L->nsp; ++s) {
        ospec *S = &L->sp[s];
        if (S->n_fo == 0) continue;
        /* Sec. 2.4.1: a0 = sum of propensities; per molecule and per own
           diffusion event the firing probability is 1 - exp(-a0 tau).      */
        double ktot = 0.0;
        for (int u = 0; u < S->n_fo; ++u) ktot += L->rx[S->fo[u]].k;
        S->T_fire = psco_threshold(-expm1(-ktot * S->tau));
        /* Eq. 5: the u-th reaction is the first whose cumulative share of a0
           reaches a0 R; integer cut points of the unit interval.            */
        double cum = 0.0;
        for (int u = 0; u < S->n_fo; ++u) {
            cum += L->rx[S->fo[u]].k;
            S->cum[u] = (u == S->n_fo - 1) ? ((uint64_t)1 << 32)
                                           : psco_threshold(ktot > 0.0 ? cum / ktot : 1.0);
        }
    }
    return clamped;
}

int psco_populate(psco_lattice *L, uint64_t seed)
{
    if (!L) return PSCO_E_ARG;
    if (L->populated) return PSCO_E_ORDER;
    int64_t N = 0;
    for (int s = 0; s < L->nsp; ++s) N += L->sp[s].n0;
    if (N > L->V) return PSCO_E_FULL;
    /* each compartment must hold its species' molecules */
    {
        int64_t room[PSCO_MAX_COMPARTMENTS] = {0}, need[PSCO_MAX_COMPARTMENTS] = {0};
        for (int64_t v = 0; v < L->V; ++v) room[vcomp(L, v)]++;
        for (int s = 0; s < L->nsp; ++s) need[L->sp[s].comp] += L->sp[s].n0;
        for (int c = 0; c < L->ncomp; ++c)
            if (need[c] > room[c]) return PSCO_E_FULL;
    }
    if (!reactions_fit_compartments(L)) return PSCO_E_UNSUPPORTED;
    L->seed = seed;
    int clamped = freeze_constants(L);

    L->occ = (uint16_t *)calloc((size_t)L->V, sizeof(uint16_t));
    L->who = (int64_t *)malloc((size_t)L->V * sizeof(int64_t));
    uint64_t *kv = (uint64_t *)malloc((size_t)L->V * sizeof(uint64_t));
    if (!L->occ || !L->who || !kv) { free(kv); return PSCO_E_NOMEM; }
    for (int64_t v = 0; v < L->V; ++v) {
        uint32_t u[4];
        draw(L, (uint32_t)v, 0u, TAG_POPULATE, u);
        kv[v] = ((uint64_t)u[0] << 32) | (uint64_t)v;
        L->who[v] = -1;
    }
    qsort(kv, (size_t)L->V, sizeof(uint64_t), cmp_u64);
    /* species in index order take the next voxels of their own compartment
       in that order (with one compartment: the next voxels) */
    int64_t cursor[PSCO_MAX_COMPARTMENTS] = {0};
    int64_t r = 0;
    for (int s = 0; s < L->nsp; ++s) {
        const int32_t c = L->sp[s].comp;
        for (int64_t a = 0; a < L->sp[s].n0; ++a, ++r) {
            int64_t m = mol_new(L);
            if (m < 0) { free(kv); return PSCO_E_NOMEM; }
            while (vcomp(L, (int64_t)(kv[cursor[c]] & 0xFFFFFFFFu)) != c) cursor[c]++;
            int32_t v = (int32_t)(kv[cursor[c]++] & 0xFFFFFFFFu);
            L->mol[m].v = v;
            L->mol[m].id = (uint32_t)r;
            L->mol[m].img[0] = L->mol[m].img[1] = L->mol[m].img[2] = 0;
            L->mol[m].species = (int16_t)s;
            L->occ[v] = (uint16_t)(s + 1);
            L->who[v] = m;
        }
        L->sp[s].dirty = 1;
    }
    free(kv);
    L->next_id = (uint32_t)N;
    L->g = 0;
    L->clock = 0.0;
    L->populated = 1;
    return clamped ? PSCO_W_PCLAMP : PSCO_OK;
}

/* ------------------------------------------------------------------------ */
/* one event                                                                  */
/* ------------------------------------------------------------------------ */
enum { K_NONE = 0, K_HOP, K_REACT, K_FIRE_INPLACE, K_FIRE2 };

typedef struct {
    int64_t  m;          /* mover                                    */
    int32_t  kind;
    int32_t  rx;         /* reaction index                           */
    int64_t  t;          /* target voxel                             */
    int16_t  wrap[3];
    int      won;
} intent;

/* direction d = floor(12 u0 / 2^32): a uniform pick among the 12 neighbours */
static int32_t pick_direction(uint32_t u0)
{
    return (int32_t)(((uint64_t)u0 * 12u) >> 32);
}

/* first-order choice (Eq. 5): smallest u with u3 < cum[u] */
static int32_t pick_first_order(const ospec *S, uint32_t u3)
{
    for (int u = 0; u < S->n_fo; ++u)
        if ((uint64_t)u3 < S->cum[u]) return S->fo[u];
    return S->fo[S->n_fo - 1];
}

/* vacant in-box neighbours of voxel v that lie in compartment c, in
   direction order; returns their count */
static int vacant_neighbors(const psco_lattice *L, int32_t v, int32_t c, int64_t tv[12], int16_t tw[12][3])
{
    int32_t ijk[3], o[3], w[3];
    int n = 0;
    decode(L, v, ijk);
    for (int d = 0; d < 12; ++d) {
        if (!psco_neighbor(L, ijk[0], ijk[1], ijk[2], d, o, w)) continue;
        int64_t t = encode(L, o);
        if (L->occ[t] != 0 || vcomp(L, t) != c) continue;
        tv[n] = t;
        tw[n][0] = (int16_t)w[0]; tw[n][1] = (int16_t)w[1]; tw[n][2] = (int16_t)w[2];
        ++n;
    }
    return n;
}

/* Decide what molecule m of species s does in event g, looking at the grid as
   it is now.  Sec. 2.4.1 (first-order test, once per diffusion event; a
   molecule that fires does not hop -- reading), Sec. 2.3 (hop to a random
   neighbour if it is vacant and in the molecule's own compartment), Sec.
   2.4.2 (collision with a registered partner reacts with probability p_AB,
   whatever the partner's compartment -- reading). */
static void decide(psco_lattice *L, int32_t s, uint32_t g, int64_t m, intent *it)
{
    const ospec *S = &L->sp[s];
    const omol *M = &L->mol[m];
    uint32_t u[4];
    draw(L, M->id, g, ((uint32_t)s << 4) | TAG_EVENT, u);
    it->m = m; it->kind = K_NONE; it->rx = -1; it->t = -1; it->won = 0;
    it->wrap[0] = it->wrap[1] = it->wrap[2] = 0;
    L->st.attempts++;

    if (S->n_fo > 0 && (uint64_t)u[2] < S->T_fire) {
        L->st.fires++;
        int32_t r = pick_first_order(S, u[3]);
        it->rx = r;
        if (L->rx[r].np < 2) { it->kind = K_FIRE_INPLACE; return; }
        int64_t tv[12]; int16_t tw[12][3];
        int c = vacant_neighbors(L, M->v, L->sp[L->rx[r].p[1]].comp, tv, tw);
        if (c == 0) return;                           /* no room: reaction fails */
        int j = (int)(((uint64_t)u[0] * (uint64_t)c) >> 32);
        it->kind = K_FIRE2;
        it->t = tv[j];
        memcpy(it->wrap, tw[j], sizeof(it->wrap));
        return;
    }

    int32_t d = pick_direction(u[0]);
    L->st.dir_count[d]++;
    int32_t ijk[3], o[3], w[3];
    decode(L, M->v, ijk);
    if (!psco_neighbor(L, ijk[0], ijk[1], ijk[2], d, o, w)) return;
    int64_t t = encode(L, o);
    uint16_t occ = L->occ[t];
    it->t = t;
    it->wrap[0] = (int16_t)w[0]; it->wrap[1] = (int16_t)w[1]; it->wrap[2] = (int16_t)w[2];
    if (occ == 0) {
        if (vcomp(L, t) == S->comp) it->kind = K_HOP;   /* else: another compartment */
        return;
    }
    int32_t partner = (int32_t)occ - 1;
    if (partner >= L->nsp) return;
    int32_t r = L->pair[s][partner];
    if (r < 0) return;                                /* occupied: hop fails     */
    L->st.collisions++;
    if ((uint64_t)u[1] < L->rx[r].T) {
        L->st.accepted++;
        it->kind = K_REACT;
        it->rx = r;
    }
}

static void add_wrap(int16_t img[3], const int16_t w[3])
{
    for (int a = 0; a < 3; ++a) img[a] = (int16_t)(img[a] + w[a]);
}

typedef struct { uint32_t parent; int64_t t; int32_t species; int16_t img[3]; } birth;

static int cmp_birth(const void *a, const void *b)
{
    uint32_t x = ((const birth *)a)->parent, y = ((const birth *)b)->parent;
    return (x > y) - (x < y);
}

/* place one new molecule (a second first-order product) at voxel t */
static int place_birth(psco_lattice *L, const birth *B, uint32_t id)
{
    int64_t n = mol_new(L);
    if (n < 0) return PSCO_E_NOMEM;
    L->mol[n].v = (int32_t)B->t;
    L->mol[n].id = id;
    memcpy(L->mol[n].img, B->img, sizeof(B->img));
    L->mol[n].species = -1;
    set_species(L, n, B->species);
    L->occ[B->t] = (uint16_t)(B->species + 1);
    L->who[B->t] = n;
    L->st.births++;
    return PSCO_OK;
}

/* Carry out a decided action.  Products of a second-order reaction: the first
   takes the partner's voxel and identity, the second the mover's (reading of
   Sec. 2.4.2, which does not say where products go); when that would put a
   product outside its compartment, the two trade places (each product always
   lands in its own compartment, and takes the identity of the reactant whose
   voxel it takes).  First-order: the first product keeps the reactant's voxel
   and identity, the second goes to the chosen vacant neighbour (Sec. 2.4.1). */
static int apply(psco_lattice *L, int32_t s, const intent *it, birth *out_birth, int *has_birth)
{
    omol *M = &L->mol[it->m];
    *has_birth = 0;
    switch (it->kind) {
    case K_HOP: {
        L->occ[M->v] = 0; L->who[M->v] = -1;
        M->v = (int32_t)it->t;
        add_wrap(M->img, it->wrap);
        L->occ[it->t] = (uint16_t)(s + 1); L->who[it->t] = it->m;
        L->st.hops++;
        break;
    }
    case K_REACT: {
        const orx *R = &L->rx[it->rx];
        int64_t pm = L->who[it->t];
        L->st.reactions2++;
        int straight = R->np == 0 ||
                       (L->sp[R->p[0]].comp == vcomp(L, it->t) &&
                        (R->np < 2 || L->sp[R->p[1]].comp == vcomp(L, M->v)));
        if (R->np == 0) {
            L->occ[it->t] = 0; L->who[it->t] = -1; set_species(L, pm, -1);
            L->occ[M->v] = 0;  L->who[M->v] = -1;  set_species(L, it->m, -1);
        } else if (R->np == 1 && straight) {
            set_species(L, pm, R->p[0]);
            L->occ[it->t] = (uint16_t)(R->p[0] + 1);
            L->occ[M->v] = 0;  L->who[M->v] = -1;  set_species(L, it->m, -1);
        } else if (R->np == 1) {
            set_species(L, it->m, R->p[0]);
            L->occ[M->v] = (uint16_t)(R->p[0] + 1);
            L->occ[it->t] = 0; L->who[it->t] = -1; set_species(L, pm, -1);
        } else {
            int32_t at_t = straight ? R->p[0] : R->p[1];
            int32_t at_m = straight ? R->p[1] : R->p[0];
            set_species(L, pm, at_t);
            L->occ[it->t] = (uint16_t)(at_t + 1);
            set_species(L, it->m, at_m);
            L->occ[M->v] = (uint16_t)(at_m + 1);
        }
        break;
    }
    case K_FIRE_INPLACE: {
        const orx *R = &L->rx[it->rx];
        L->st.reactions1++;
        if (R->np == 0) {
            L->occ[M->v] = 0; L->who[M->v] = -1; set_species(L, it->m, -1);
        } else {
            set_species(L, it->m, R->p[0]);
            L->occ[M->v] = (uint16_t)(R->p[0] + 1);
        }
        break;
    }
    case K_FIRE2: {
        const orx *R = &L->rx[it->rx];
        L->st.reactions1++;
        set_species(L, it->m, R->p[0]);
        L->occ[M->v] = (uint16_t)(R->p[0] + 1);
        out_birth->parent = M->id;
        out_birth->t = it->t;
        out_birth->species = R->p[1];
        memcpy(out_birth->img, M->img, sizeof(M->img));
        add_wrap(out_birth->img, it->wrap);
        *has_birth = 1;
        break;
    }
    default:
        break;
    }
    return PSCO_OK;
}

typedef struct { int64_t t; uint32_t id; int64_t k; } claim;

static int cmp_claim(const void *a, const void *b)
{
    const claim *x = (const claim *)a, *y = (const claim *)b;
    if (x->t != y->t) return (x->t > y->t) - (x->t < y->t);
    return (x->id > y->id) - (x->id < y->id);
}

/* synchronous rule: decide all against the grid at the start of the event,
   the lowest id wins each contested target, then carry out the winners */
static int event_sync(psco_lattice *L, int32_t s, uint32_t g)
{
    int rc = rebuild_list(L, s);
    if (rc) return rc;
    int64_t n = L->sp[s].nlist;
    if (n == 0) return PSCO_OK;
    intent *it = (intent *)malloc((size_t)n * sizeof(intent));
    claim *cl = (claim *)malloc((size_t)n * sizeof(claim));
    birth *br = (birth *)malloc((size_t)n * sizeof(birth));
    if (!it || !cl || !br) { free(it); free(cl); free(br); return PSCO_E_NOMEM; }

    for (int64_t a = 0; a < n; ++a) decide(L, s, g, L->sp[s].list[a], &it[a]);

    int64_t nc = 0;
    for (int64_t a = 0; a < n; ++a) {
        if (it[a].kind == K_HOP || it[a].kind == K_REACT || it[a].kind == K_FIRE2) {
            cl[nc].t = it[a].t; cl[nc].id = L->mol[it[a].m].id; cl[nc].k = a; ++nc;
        } else if (it[a].kind == K_FIRE_INPLACE) {
            it[a].won = 1;                       /* needs no voxel */
        }
    }
    qsort(cl, (size_t)nc, sizeof(claim), cmp_claim);
    for (int64_t a = 0; a < nc; ++a)
        if (a == 0 || cl[a].t != cl[a - 1].t) it[cl[a].k].won = 1;

    int64_t nb = 0;
    for (int64_t a = 0; a < n; ++a) {
        if (!it[a].won) continue;
        int hb = 0;
        apply(L, s, &it[a], &br[nb], &hb);
        nb += hb;
    }
    /* fresh ids go to the successful parents in ascending parent-id order */
    qsort(br, (size_t)nb, sizeof(birth), cmp_birth);
    for (int64_t a = 0; a < nb && rc == PSCO_OK; ++a)
        rc = place_birth(L, &br[a], L->next_id++);
    free(it); free(cl); free(br);
    return rc;
}

/* the paper's one-by-one update (Sec. 2.3): each molecule sees the grid as
   left by the molecules before it; order ascending id, or a fresh random
   permutation of that list */
static int event_seq(psco_lattice *L, int32_t s, uint32_t g, int random_order)
{
    int rc = rebuild_list(L, s);
    if (rc) return rc;
    int64_t n = L->sp[s].nlist;
    if (n == 0) return PSCO_OK;
    int64_t *order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!order) return PSCO_E_NOMEM;
    memcpy(order, L->sp[s].list, (size_t)n * sizeof(int64_t));
    if (random_order) {                           /* Fisher-Yates */
        for (int64_t a = n - 1; a > 0; --a) {
            uint32_t u[4];
            draw(L, (uint32_t)a, g, ((uint32_t)s << 4) | TAG_ORDER, u);
            int64_t b = (int64_t)(((uint64_t)u[0] * (uint64_t)(a + 1)) >> 32);
            int64_t tmp = order[a]; order[a] = order[b]; order[b] = tmp;
        }
    }
    for (int64_t a = 0; a < n && rc == PSCO_OK; ++a) {
        intent it;
        decide(L, s, g, order[a], &it);
        birth b; int hb = 0;
        apply(L, s, &it, &b, &hb);
        if (hb) rc = place_birth(L, &b, L->next_id++);
    }
    free(order);
    return rc;
}

/* the paper's sub-volume scheme (Sec. 2.5: sub-volumes are taken one after
   another in a random order, so that those processed at the same time never
   touch each other), on the lattice: sub-volumes of 2 x 2 x 2 voxels, colour
   = parities of the sub-volume indices (i/2, j/2, k/2).  Sub-volumes of one
   colour are at least one sub-volume apart, so a hop (one voxel) from one of
   them never reaches what a hop from another reads or writes.  The event's
   colour order is a Fisher-Yates shuffle of 0..7 with draw (a, g, s<<4 |
   TAG_SUBVOL) for a = 7..1; each colour takes, in ascending id, the molecules
   of the species standing in its sub-volumes that the event has not yet
   processed, each seeing the grid as left before it. */
static int subvol_colour(const psco_lattice *L, int64_t v)
{
    int32_t c[3];
    decode(L, v, c);
    return ((c[0] >> 1) & 1) | (((c[1] >> 1) & 1) << 1) | (((c[2] >> 1) & 1) << 2);
}

static int event_subvol(psco_lattice *L, int32_t s, uint32_t g)
{
    int rc = rebuild_list(L, s);
    if (rc) return rc;
    int64_t n = L->sp[s].nlist;
    if (n == 0) return PSCO_OK;
    int64_t *order = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    unsigned char *done = (unsigned char *)calloc((size_t)n, 1);
    if (!order || !done) { free(order); free(done); return PSCO_E_NOMEM; }
    memcpy(order, L->sp[s].list, (size_t)n * sizeof(int64_t));
    int colours[8] = {0, 1, 2, 3, 4, 5, 6, 7};
    for (int a = 7; a > 0; --a) {
        uint32_t u[4];
        draw(L, (uint32_t)a, g, ((uint32_t)s << 4) | TAG_SUBVOL, u);
        int b = (int)(((uint64_t)u[0] * (uint64_t)(a + 1)) >> 32);
        int tmp = colours[a]; colours[a] = colours[b]; colours[b] = tmp;
    }
    for (int ci = 0; ci < 8 && rc == PSCO_OK; ++ci) {
        for (int64_t a = 0; a < n && rc == PSCO_OK; ++a) {
            if (done[a] || subvol_colour(L, L->mol[order[a]].v) != colours[ci]) continue;
            done[a] = 1;
            intent it;
            decide(L, s, g, order[a], &it);
            birth b; int hb = 0;
            apply(L, s, &it, &b, &hb);
            if (hb) rc = place_birth(L, &b, L->next_id++);
        }
    }
    free(order);
    free(done);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* event scheduler (Sec. 2.2): the next event is the mobile species with the  */
/* earliest next diffusion time (events_done + 1) * tau; ties go to the lower  */
/* species index.  Immobile species have no events.                           */
/* ------------------------------------------------------------------------ */
static int next_event(const psco_lattice *L, int32_t *s_out, double *t_out)
{
    int32_t best = -1;
    double tb = 0.0;
    for (int32_t s = 0; s < L->nsp; ++s) {
        if (!(L->sp[s].D > 0.0)) continue;
        double t = (double)(L->sp[s].done + 1) * L->sp[s].tau;
        if (best < 0 || t < tb) { best = s; tb = t; }
    }
    *s_out = best;
    *t_out = tb;
    return best >= 0;
}

static int do_event(psco_lattice *L, int32_t s)
{
    if (L->g == UINT32_MAX) return PSCO_E_LIMIT;
    int rc;
    if (L->rule == PSCO_RULE_SYNC) rc = event_sync(L, s, L->g);
    else if (L->rule == PSCO_RULE_SUBVOL) rc = event_subvol(L, s, L->g);
    else rc = event_seq(L, s, L->g, L->rule == PSCO_RULE_SEQ_RANDOM);
    if (rc) return rc;
    L->sp[s].done++;
    L->g++;
    L->st.events++;
    return PSCO_OK;
}

int psco_run(psco_lattice *L, double t_end)
{
    if (!L || isnan(t_end) || isinf(t_end)) return PSCO_E_ARG;
    if (!L->populated) return PSCO_E_ORDER;
    for (;;) {
        int32_t s; double t;
        if (!next_event(L, &s, &t) || t > t_end) break;
        int rc = do_event(L, s);
        if (rc) return rc;
        L->clock = t;
    }
    if (t_end > L->clock) L->clock = t_end;
    return PSCO_OK;
}

int psco_run_events(psco_lattice *L, int64_t n_events)
{
    if (!L || n_events < 0) return PSCO_E_ARG;
    if (!L->populated) return PSCO_E_ORDER;
    for (int64_t e = 0; e < n_events; ++e) {
        int32_t s; double t;
        if (!next_event(L, &s, &t)) break;
        int rc = do_event(L, s);
        if (rc) return rc;
        L->clock = t;
    }
    return PSCO_OK;
}

/* ------------------------------------------------------------------------ */
/* read-out                                                                   */
/* ------------------------------------------------------------------------ */
int psco_counts(const psco_lattice *L, int64_t *counts, int32_t n)
{
    if (!L || !counts || n < L->nsp) return PSCO_E_ARG;
    for (int s = 0; s < n; ++s) counts[s] = 0;
    for (int64_t m = 0; m < L->nmol; ++m)
        if (L->mol[m].species >= 0) counts[L->mol[m].species]++;
    return PSCO_OK;
}

static int collect(const psco_lattice *L, int32_t s, int64_t **out, int64_t *n_out)
{
    int64_t n = 0;
    for (int64_t m = 0; m < L->nmol; ++m) if (L->mol[m].species == s) ++n;
    int64_t *lst = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!lst) return PSCO_E_NOMEM;
    n = 0;
    for (int64_t m = 0; m < L->nmol; ++m) if (L->mol[m].species == s) lst[n++] = m;
    g_sort_ctx = L;
    qsort(lst, (size_t)n, sizeof(int64_t), cmp_index_by_id);
    *out = lst; *n_out = n;
    return PSCO_OK;
}

int psco_coords(const psco_lattice *L, int32_t s, int32_t *ijk, uint32_t *ids,
                int64_t cap, int64_t *n_out)
{
    if (!L || !n_out || s < 0 || s >= L->nsp) return PSCO_E_ARG;
    if (!L->populated) return PSCO_E_ORDER;
    int64_t *lst, n;
    int rc = collect(L, s, &lst, &n);
    if (rc) return rc;
    *n_out = n;
    if (n > cap || (n > 0 && !ijk)) { free(lst); return PSCO_E_ARG; }
    for (int64_t a = 0; a < n; ++a) {
        decode(L, L->mol[lst[a]].v, &ijk[3 * a]);
        if (ids) ids[a] = L->mol[lst[a]].id;
    }
    free(lst);
    return PSCO_OK;
}

/* unwrapped integer basis: X = 2I + P, Y = 3J + (K & 1), Z = K with
   I = i + img_i N_i (likewise J, K) and P = (J + K) & 1; the centre is then
   (X, Y / sqrt(3), Z * 2 sqrt(2/3)) in units of r_v.  FCC: Y = 3J + (K mod 3)
   and P = (J + [K mod 3 == 1]) & 1. */
int psco_unwrapped(const psco_lattice *L, int32_t s, int32_t *xyz, uint32_t *ids,
                   int64_t cap, int64_t *n_out)
{
    if (!L || !n_out || s < 0 || s >= L->nsp) return PSCO_E_ARG;
    if (!L->populated) return PSCO_E_ORDER;
    int64_t *lst, n;
    int rc = collect(L, s, &lst, &n);
    if (rc) return rc;
    *n_out = n;
    if (n > cap || (n > 0 && !xyz)) { free(lst); return PSCO_E_ARG; }
    for (int64_t a = 0; a < n; ++a) {
        const omol *M = &L->mol[lst[a]];
        int32_t c[3];
        decode(L, M->v, c);
        int32_t I = c[0] + (int32_t)M->img[0] * L->ni;
        int32_t J = c[1] + (int32_t)M->img[1] * L->nj;
        int32_t K = c[2] + (int32_t)M->img[2] * L->nk;
        if (L->bflags & PSCO_FCC) {
            int32_t c3 = ((K % 3) + 3) % 3;
            xyz[3 * a + 0] = 2 * I + ((J + (c3 == 1)) & 1);
            xyz[3 * a + 1] = 3 * J + c3;
        } else {
            xyz[3 * a + 0] = 2 * I + ((J + K) & 1);
            xyz[3 * a + 1] = 3 * J + (K & 1);
        }
        xyz[3 * a + 2] = K;
        if (ids) ids[a] = M->id;
    }
    free(lst);
    return PSCO_OK;
}

int psco_grid(const psco_lattice *L, uint16_t *occ)
{
    if (!L || !occ) return PSCO_E_ARG;
    if (!L->populated) return PSCO_E_ORDER;
    memcpy(occ, L->occ, (size_t)L->V * sizeof(uint16_t));
    return PSCO_OK;
}

int psco_time(const psco_lattice *L, double *t)
{
    if (!L || !t) return PSCO_E_ARG;
    *t = L->clock;
    return PSCO_OK;
}

int psco_event_index(const psco_lattice *L, uint32_t *g)
{
    if (!L || !g) return PSCO_E_ARG;
    *g = L->g;
    return PSCO_OK;
}

int psco_stats_get(const psco_lattice *L, psco_stats *s)
{
    if (!L || !s) return PSCO_E_ARG;
    *s = L->st;
    return PSCO_OK;
}

int psco_place(psco_lattice *L, int32_t s, int32_t v, uint32_t *id_out)
{
    if (!L || s < 0 || s >= L->nsp || v < 0 || v >= L->V) return PSCO_E_ARG;
    if (!L->populated) return PSCO_E_ORDER;
    if (L->occ[v] != 0) return PSCO_E_FULL;
    if (vcomp(L, v) != L->sp[s].comp) return PSCO_E_ARG;
    int64_t m = mol_new(L);
    if (m < 0) return PSCO_E_NOMEM;
    L->mol[m].v = v;
    L->mol[m].id = L->next_id++;
    L->mol[m].img[0] = L->mol[m].img[1] = L->mol[m].img[2] = 0;
    L->mol[m].species = -1;
    set_species(L, m, s);
    L->occ[v] = (uint16_t)(s + 1);
    L->who[v] = m;
    if (id_out) *id_out = L->mol[m].id;
    return PSCO_OK;
}

/* grid, voxel owner table and molecule records must agree exactly */
int psco_check(const psco_lattice *L)
{
    if (!L || !L->populated) return PSCO_E_ARG;
    for (int64_t v = 0; v < L->V; ++v) {
        int64_t m = L->who[v];
        if ((L->occ[v] == 0) != (m < 0)) return 1;
        if (m >= 0) {
            if (m >= L->nmol) return 2;
            if (L->mol[m].v != v) return 3;
            if (L->mol[m].species + 1 != L->occ[v]) return 4;
            if (L->sp[L->mol[m].species].comp != vcomp(L, v)) return 6;
        }
    }
    for (int64_t m = 0; m < L->nmol; ++m) {
        if (L->mol[m].species < 0) continue;
        if (L->who[L->mol[m].v] != m) return 5;
    }
    return 0;
}
