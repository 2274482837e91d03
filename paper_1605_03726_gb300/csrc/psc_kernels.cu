// psc_kernels.cu -- sm_103a kernels of one species event (Sec. 2.2-2.4 of
// Miyauchi et al., arXiv:1605.03726) under the synchronous conflict rule.
//
// An event of species s runs as
//   claim    every molecule draws (Philox), takes its first-order test, picks a
//            neighbour, reads the grid as it was at the start of the event and,
//            if the neighbour is vacant (or holds a partner and the collision is
//            accepted), claims it: the claim slot of a voxel keeps the lowest id;
//   commit   each winner writes the grid (move, reaction products, first-order
//            products);
//   reconcile   (only for species touched by reactions) lists are brought back
//            in line with the grid: an entry whose voxel now holds another
//            species moves to that species' list, an emptied one is dropped;
//   births   fresh ids for second first-order products, in parent-id order.
// The hot path of a diffusion-only species is claim + commit.
//
// Grid state.  Vacancy lives in a 1-bit-per-voxel mirror (16.8 MB at 512^3, so
// it stays in L2); the 16-bit species codes are kept exact for every species
// that takes part in a reaction.  A species without reactions skips the code
// writes while it moves: nothing reads its codes before a read-out, which
// rebuilds them from its list.  Claims go to a per-voxel word on small
// lattices and to a compact hash table (two slots per molecule) on large ones,
// so the claim traffic of an event touches a few MB instead of random words
// of a V-sized array.
#include "psc_internal.h"

#include <algorithm>
#include <climits>

namespace psc {

// HCP stencil in twisted Cartesian coordinates (Sec. 2.1): for directions
// d = 0..11 the offsets (di, dj, dk) + 1 packed in 2-bit fields.  di depends on
// the parity p = (j + k) & 1, dj on the parity of k, dk on nothing:
//   d  0: ( +1,  0,  0)        d  6: (p-1,  0, -1)
//   d  1: ( -1,  0,  0)        d  7: ( p ,  0, -1)
//   d  2: (p-1, -1,  0)        d  8: (  0, dz, -1)   dz = +1 for odd k, -1 for even k
//   d  3: ( p , -1,  0)        d  9: (p-1,  0, +1)
//   d  4: (p-1, +1,  0)        d 10: ( p ,  0, +1)
//   d  5: ( p , +1,  0)        d 11: (  0, dz, +1)
// Words: [0] di for p = 0, [1] di for p = 1, [2] dj for even k, [3] dj for odd
// k, [4] dk.  Every warp reads all five words (uniform addresses), then picks
// per thread, so the constant cache serves them as broadcasts.
// FCC lattice (App. B; ABC stacking, c = k mod 3, p = (j + [c == 1]) & 1):
// the same di and dk words; dj from words [5 + c]:
//   d 6, 7: a = -1 for c = 0, else 0     d 8:  b = 0 for c = 0, else +1
//   d 9,10: a' = +1 for c = 2, else 0    d 11: b' = 0 for c = 2, else -1
__constant__ uint32_t c_stencil[8];

static uint32_t pack_offsets(const int (&o)[12])
{
    uint32_t w = 0;
    for (int d = 0; d < 12; ++d) w |= (uint32_t)(o[d] + 1) << (2 * d);
    return w;
}

void upload_stencil(cudaStream_t st)
{
    const int di0[12] = {+1, -1, -1, 0, -1, 0, -1, 0, 0, -1, 0, 0};
    const int di1[12] = {+1, -1, 0, +1, 0, +1, 0, +1, 0, 0, +1, 0};
    const int dj0[12] = {0, 0, -1, -1, +1, +1, 0, 0, -1, 0, 0, -1};
    const int dj1[12] = {0, 0, -1, -1, +1, +1, 0, 0, +1, 0, 0, +1};
    const int dk[12] = {0, 0, 0, 0, 0, 0, -1, -1, -1, +1, +1, +1};
    const int fj0[12] = {0, 0, -1, -1, +1, +1, -1, -1, 0, 0, 0, -1};
    const int fj1[12] = {0, 0, -1, -1, +1, +1, 0, 0, +1, 0, 0, -1};
    const int fj2[12] = {0, 0, -1, -1, +1, +1, 0, 0, +1, +1, +1, 0};
    static uint32_t h[8];
    h[0] = pack_offsets(di0); h[1] = pack_offsets(di1);
    h[2] = pack_offsets(dj0); h[3] = pack_offsets(dj1);
    h[4] = pack_offsets(dk);
    h[5] = pack_offsets(fj0); h[6] = pack_offsets(fj1); h[7] = pack_offsets(fj2);
    cudaMemcpyToSymbolAsync(c_stencil, h, sizeof(h), 0, cudaMemcpyHostToDevice, st);
}

// Compact Morton code: level by level from the least significant bit, the
// next bit of i, of j, of k in turn, skipping an axis once its extent is used
// up; codes wider than 32 bits keep their top 32.
void build_morton_tables(int32_t ni, int32_t nj, int32_t nk, uint32_t* out, uint32_t* bits_out)
{
    const int32_t n[3] = {ni, nj, nk};
    int nb[3];
    for (int a = 0; a < 3; ++a) {
        nb[a] = 0;
        while ((1ll << nb[a]) < n[a]) ++nb[a];
    }
    int pos[3][32];
    int total = 0;
    const int levels = std::max(nb[0], std::max(nb[1], nb[2]));
    for (int l = 0; l < levels; ++l)
        for (int a = 0; a < 3; ++a)
            if (l < nb[a]) pos[a][l] = total++;
    const int drop = total > 32 ? total - 32 : 0;
    uint32_t* dst = out;
    for (int a = 0; a < 3; ++a) {
        for (int32_t x = 0; x < n[a]; ++x) {
            uint64_t c = 0;
            for (int l = 0; l < nb[a]; ++l)
                if ((x >> l) & 1) c |= 1ull << pos[a][l];
            *dst++ = (uint32_t)(c >> drop);
        }
    }
    *bits_out = (uint32_t)(total - drop);
}

FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    if (d <= 1) { f.m = 0; f.s = -1; return f; }
    int l = 0;
    while ((1ull << l) < d) ++l;                       // l = ceil(log2 d)
    const unsigned p = 31u + (unsigned)l;
    f.m = (uint32_t)(((1ull << p) + d - 1) / d);      // ceil(2^p / d) < 2^32
    f.s = (int32_t)(p - 32u);
    return f;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f)
{
    return f.s < 0 ? n : (__umulhi(n, f.m) >> f.s);
}

__device__ __forceinline__ void decode(const Geometry& G, uint32_t v, int32_t& i, int32_t& j, int32_t& k)
{
    const uint32_t kk = fdiv(v, G.div_ninj);
    const uint32_t r = v - kk * G.ninj;
    const uint32_t jj = fdiv(r, G.div_ni);
    i = (int32_t)(r - jj * (uint32_t)G.ni);
    j = (int32_t)jj;
    k = (int32_t)kk;
}

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1, uint32_t (&u)[4])
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c2 = hi0 ^ c3 ^ k1;
        c1 = lo1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    u[0] = c0; u[1] = c1; u[2] = c2; u[3] = c3;
}

// neighbour of a voxel: linear index, coordinates, change of the wrap counters
struct Nb {
    int32_t t, i, j, k;
    uint64_t wrap;
};

// Neighbour d of (i, j, k); false if it lies behind a reflective wall.
__device__ __forceinline__ bool neighbor(const Geometry& G, int32_t i, int32_t j, int32_t k, int d, Nb& nb)
{
    const uint32_t s0 = c_stencil[0], s1 = c_stencil[1], s2 = c_stencil[2], s3 = c_stencil[3],
                   s4 = c_stencil[4];
    uint32_t wi, wj;
    if (G.bflags & 8u) {                          // FCC
        const int c = k % 3;
        const uint32_t f0 = c_stencil[5], f1 = c_stencil[6], f2 = c_stencil[7];
        wi = ((j + (c == 1 ? 1 : 0)) & 1) ? s1 : s0;
        wj = c == 0 ? f0 : (c == 1 ? f1 : f2);
    } else {
        wi = ((j + k) & 1) ? s1 : s0;
        wj = (k & 1) ? s3 : s2;
    }
    int32_t ti = i + (int32_t)((wi >> (2 * d)) & 3u) - 1;
    int32_t tj = j + (int32_t)((wj >> (2 * d)) & 3u) - 1;
    int32_t tk = k + (int32_t)((s4 >> (2 * d)) & 3u) - 1;
    uint64_t w = 0;
    if (ti < 0) {
        if (!(G.bflags & 1u)) return false;
        ti += G.ni; w |= 0xFFFFull;
    } else if (ti >= G.ni) {
        if (!(G.bflags & 1u)) return false;
        ti -= G.ni; w |= 0x1ull;
    }
    if (tj < 0) {
        if (!(G.bflags & 2u)) return false;
        tj += G.nj; w |= 0xFFFFull << 16;
    } else if (tj >= G.nj) {
        if (!(G.bflags & 2u)) return false;
        tj -= G.nj; w |= 0x1ull << 16;
    }
    if (tk < 0) {
        if (!(G.bflags & 4u)) return false;
        tk += G.nk; w |= 0xFFFFull << 32;
    } else if (tk >= G.nk) {
        if (!(G.bflags & 4u)) return false;
        tk -= G.nk; w |= 0x1ull << 32;
    }
    nb.t = ti + G.ni * (tj + G.nj * tk);
    nb.i = ti; nb.j = tj; nb.k = tk;
    nb.wrap = w;
    return true;
}

// fieldwise 16-bit add of packed wrap counters (no carry between fields)
__device__ __forceinline__ uint64_t img_add(uint64_t a, uint64_t b)
{
    const uint64_t H = 0x0000800080008000ull;
    return ((a & ~H) + (b & ~H)) ^ ((a ^ b) & H);
}

__device__ __forceinline__ int pick_first_order(const ModelDev* M, int s, uint32_t u3)
{
    const int n = M->n_fo[s];
    for (int u = 0; u < n - 1; ++u)
        if ((uint64_t)u3 < M->fo_cum[s][u]) return M->fo_rx[s][u];
    return M->fo_rx[s][n - 1];
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ void flush_stat(unsigned long long* dst, unsigned long long v)
{
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// ---------------------------------------------------------------------------
// vacancy mirror: one bit per voxel, words are 4 x 4 x 2 bricks (i, j, k) so a
// hop often stays inside one word and flips both bits with one atomicXor
// ---------------------------------------------------------------------------
struct BitPos {
    uint32_t word, mask;
};

__device__ __forceinline__ BitPos bitpos(const Geometry& G, int32_t i, int32_t j, int32_t k)
{
    BitPos b;
    b.word = (((uint32_t)k >> 1) * G.nbj + ((uint32_t)j >> 2)) * G.nbi + ((uint32_t)i >> 2);
    b.mask = 1u << (((uint32_t)i & 3u) | (((uint32_t)j & 3u) << 2) | (((uint32_t)k & 1u) << 4));
    return b;
}

__device__ __forceinline__ bool occupied(const uint32_t* bits, BitPos b)
{
    return (__ldcg(&bits[b.word]) & b.mask) != 0u;
}

__device__ __forceinline__ void bit_set(uint32_t* bits, BitPos b) { atomicOr(&bits[b.word], b.mask); }
__device__ __forceinline__ void bit_clear(uint32_t* bits, BitPos b) { atomicAnd(&bits[b.word], ~b.mask); }

// a molecule leaves `from` (set) for `to` (clear)
__device__ __forceinline__ void bit_move(uint32_t* bits, BitPos from, BitPos to)
{
    if (from.word == to.word) {
        atomicXor(&bits[from.word], from.mask | to.mask);
    } else {
        atomicAnd(&bits[from.word], ~from.mask);
        atomicOr(&bits[to.word], to.mask);
    }
}

// ---------------------------------------------------------------------------
// claim tables
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t morton(const Geometry& G, int32_t i, int32_t j, int32_t k)
{
    return __ldg(&G.mort[i]) | __ldg(&G.mort[G.ni + j]) | __ldg(&G.mort[G.ni + G.nj + k]);
}

// Home slot of voxel t = (i, j, k).  Map 0: Fibonacci hash of t (claims spread
// over the whole table).  Map 1: the compact Morton code scaled to the table,
// so molecules handled together (a stretch of the Morton-sorted list) claim a
// compact region of it.  Map 2: as 1, with the low 10 bits permuted (odd
// multiplier mod 1024) so neighbouring claims land on different cache lines.
__device__ __forceinline__ uint32_t slot_of(const Geometry& G, uint32_t t, int32_t i, int32_t j, int32_t k,
                                            uint32_t hash_bits)
{
    if (G.slot_map == 0u) return (t * 2654435761u) >> (32u - hash_bits);
    const uint32_t c = morton(G, i, j, k);
    uint32_t h = G.mort_bits >= hash_bits ? c >> (G.mort_bits - hash_bits) : c << (hash_bits - G.mort_bits);
    if (G.slot_map == 2u && hash_bits > 10u) h = (h & ~0x3FFu) | ((h * 0x2C9u) & 0x3FFu);
    return h;
}

// Claim voxel t = (i, j, k) for molecule id in an open-addressing table of
// 2^hash_bits slots, starting at slot h whose content is believed to be cur;
// the slot of t ends up holding the lowest id.  Returns the slot, or -1 if the
// table is full (error raised).
__device__ __forceinline__ int32_t hash_claim_from(uint64_t* tab, uint32_t hash_bits, uint32_t t, uint32_t id,
                                                   uint32_t h, uint64_t cur, int32_t* err)
{
    const uint32_t mask = (1u << hash_bits) - 1u;
    const uint64_t mine = ((uint64_t)t << 32) | id;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        if (cur == kEmptySlot) {
            const unsigned long long prev = atomicCAS((unsigned long long*)&tab[h],
                                                      (unsigned long long)kEmptySlot, (unsigned long long)mine);
            if (prev == kEmptySlot) return (int32_t)h;
            cur = prev;
        }
        if ((uint32_t)(cur >> 32) == t) {
            // same voxel: a slot's key never changes within the event, so the
            // 64-bit minimum is the minimum over ids
            if ((uint32_t)cur > id) atomicMin((unsigned long long*)&tab[h], (unsigned long long)mine);
            return (int32_t)h;
        }
        h = (h + 1u) & mask;
        cur = __ldcg((const unsigned long long*)&tab[h]);
    }
    atomicOr(err, kErrClaimTableFull);
    return -1;
}

__device__ __forceinline__ int32_t hash_claim(const Geometry& G, uint64_t* tab, uint32_t hash_bits, const Nb& nb,
                                              uint32_t id, int32_t* err)
{
    const uint32_t h = slot_of(G, (uint32_t)nb.t, nb.i, nb.j, nb.k, hash_bits);
    return hash_claim_from(tab, hash_bits, (uint32_t)nb.t, id, h,
                           __ldcg((const unsigned long long*)&tab[h]), err);
}

template <bool HASH>
__device__ __forceinline__ void claim(const EventArgs& a, const Nb& nb, uint32_t id)
{
    if (HASH) hash_claim(a.geo, a.ct.hash, a.ct.hash_bits, nb, id, &a.sc->err);
    else atomicMin(&a.ct.direct[nb.t], id);
}

// Did molecule id win voxel nb?  (Direct mode: the winner resets the word,
// which every loser then reads as "not mine".)
template <bool HASH>
__device__ __forceinline__ bool won(const EventArgs& a, const Nb& nb, uint32_t id)
{
    const uint32_t t = (uint32_t)nb.t;
    if (!HASH) {
        if (a.ct.direct[t] != id) return false;
        a.ct.direct[t] = kNoClaim;
        return true;
    }
    const uint32_t mask = (1u << a.ct.hash_bits) - 1u;
    uint32_t h = slot_of(a.geo, t, nb.i, nb.j, nb.k, a.ct.hash_bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint64_t cur = __ldcg((const unsigned long long*)&a.ct.hash[h]);
        if (cur == kEmptySlot) return false;
        if ((uint32_t)(cur >> 32) == t) return (uint32_t)cur == id;
        h = (h + 1u) & mask;
    }
    return false;
}

// the mirror word (4 x 4 x 2 brick) holding a voxel whose species changed:
// the reconcile passes re-check only list entries in such bricks
__device__ __forceinline__ void mark_dirty(uint32_t* dirty, uint32_t word)
{
    atomicOr(&dirty[word >> 5], 1u << (word & 31u));
}

// ---------------------------------------------------------------------------
// claim
// ---------------------------------------------------------------------------
// The body of each event kernel takes its block index and block count
// explicitly, so a batched launch can hand each replica a range of blocks.
template <bool GENERAL, bool HASH>
__device__ __forceinline__ void claim_body(const EventArgs& a, uint32_t g, int blk, int nblk)
{
    const int32_t n = *a.count;
    if (blk == 0 && threadIdx.x < kMaxSpecies) a.sc->tmp_count[threadIdx.x] = 0;
    unsigned long long n_att = 0, n_col = 0, n_acc = 0, n_fire = 0;
    const uint32_t c2 = ((uint32_t)a.s << 4) | kTagEvent;
    const int stride = nblk * blockDim.x;
    for (int base = blk * blockDim.x; base < n; base += stride) {
        const int idx = base + threadIdx.x;
        if (idx >= n) continue;
        const uint32_t v = (uint32_t)a.list.vox[idx];
        const uint32_t id = a.list.ids[idx];
        int32_t i, j, k;
        decode(a.geo, v, i, j, k);
        uint32_t u[4];
        philox(id, g, c2, 0u, a.key0, a.key1, u);
        ++n_att;
        uint8_t out = kDecNone;
        if (GENERAL) {
            const ModelDev* M = a.model;
            if (M->n_fo[a.s] > 0 && (uint64_t)u[2] < M->T_fire[a.s]) {
                ++n_fire;
                if (a.dec) a.dec[idx] = kDecFire;
                const int r = pick_first_order(M, a.s, u[3]);
                if (M->rx[r].np == 2) {
                    // second product: uniform pick among neighbours vacant now
                    // in its compartment (clear in its compartment's mirror)
                    const uint32_t* pb = M->mirror[M->rx[r].p1];
                    int c = 0;
                    for (int d = 0; d < 12; ++d) {
                        Nb nb;
                        if (neighbor(a.geo, i, j, k, d, nb) && !occupied(pb, bitpos(a.geo, nb.i, nb.j, nb.k))) ++c;
                    }
                    if (c > 0) {
                        int want = (int)__umulhi(u[0], (uint32_t)c);
                        for (int d = 0; d < 12; ++d) {
                            Nb nb;
                            if (neighbor(a.geo, i, j, k, d, nb) && !occupied(pb, bitpos(a.geo, nb.i, nb.j, nb.k))) {
                                if (want == 0) { claim<HASH>(a, nb, id); break; }
                                --want;
                            }
                        }
                    }
                }
                continue;
            }
        }
        const int d = (int)__umulhi(u[0], 12u);
        Nb nb;
        if (neighbor(a.geo, i, j, k, d, nb)) {
            if (!occupied(a.bits, bitpos(a.geo, nb.i, nb.j, nb.k))) {
                claim<HASH>(a, nb, id);
                out = (uint8_t)d;
            } else if (GENERAL) {
                const uint16_t o = a.occ[nb.t];
                if (o != 0 && o != kBlocked) {
                    const int r = a.model->pair[a.s][o - 1];
                    if (r >= 0) {
                        ++n_col;
                        if ((uint64_t)u[1] < a.model->rx[r].T) {
                            ++n_acc;
                            claim<HASH>(a, nb, id);
                            out = (uint8_t)d;
                        }
                    }
                }
            }
        }
        if (a.dec) a.dec[idx] = out;
    }
    if (a.collect_stats) {
        flush_stat(&a.sc->stats[kStatAttempts], n_att);
        if (GENERAL) {
            flush_stat(&a.sc->stats[kStatCollisions], n_col);
            flush_stat(&a.sc->stats[kStatAccepted], n_acc);
            flush_stat(&a.sc->stats[kStatFires], n_fire);
        }
    }
}

// the event index: in a replayed graph, the graph's first index plus the
// event's place in it
__device__ __forceinline__ uint32_t event_index(const EventArgs& a)
{
    return a.g_base ? __ldcg(a.g_base) + a.g : a.g;
}

template <bool GENERAL, bool HASH>
__global__ void __launch_bounds__(256) k_claim(const EventArgs a)
{
    claim_body<GENERAL, HASH>(a, event_index(a), blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// commit
// ---------------------------------------------------------------------------
// The mover at list slot idx (voxel v) now stands as species code nc on its
// voxel (0: gone).  Unless it is still the due species, its entry leaves the
// list (slot noted for the fill pass, voxel marked -1) and, for a product,
// joins the product's list with its id and wrap counters.  Only a molecule's
// own action changes an entry of the due species' list, so this replaces the
// list's check against the grid.
__device__ __forceinline__ void mover_leaves(const EventArgs& a, int idx, uint32_t v, uint32_t id, uint16_t nc)
{
    if (nc == (uint16_t)(a.s + 1)) return;
    const int slot = atomicAdd(&a.sc->tmp_count[a.s], 1);
    a.leave[slot] = idx;
    const uint64_t img = a.list.img[idx];
    a.list.vox[idx] = -1;
    if (nc == 0 || nc == kBlocked) return;
    const int y = (int)nc - 1;
    const SpeciesList dst = a.model->lists[y];
    const int s2 = atomicAdd(&a.sc->counts[y], 1);
    if (s2 < dst.cap) {
        dst.vox[s2] = (int32_t)v;
        dst.ids[s2] = id;
        dst.img[s2] = img;
    } else {
        atomicOr(&a.sc->err, kErrListOverflow);
    }
}

template <bool GENERAL, bool HASH>
__device__ __forceinline__ void commit_body(const EventArgs& a, uint32_t g, int blk, int nblk)
{
    const int32_t n = *a.count;
    unsigned long long n_hop = 0, n_r2 = 0, n_r1 = 0;
    const uint32_t c2 = ((uint32_t)a.s << 4) | kTagEvent;
    const uint16_t self = (uint16_t)(a.s + 1);
    const int stride = nblk * blockDim.x;
    if (HASH) {
        // empty the table of the previous event for the next one
        for (uint32_t x = blk * blockDim.x + threadIdx.x; x < a.ct.clear_n; x += stride)
            a.ct.clear[x] = kEmptySlot;
    }
    uint32_t* dirty = a.dirty[g & 1u];
    if (GENERAL) {
        // the previous event's map is read; empty it for the next one
        uint32_t* old = a.dirty[(g & 1u) ^ 1u];
        for (uint32_t x = blk * blockDim.x + threadIdx.x; x < a.dirty_words; x += stride) old[x] = 0u;
    }
    for (int base = blk * blockDim.x; base < n; base += stride) {
        const int idx = base + threadIdx.x;
        if (idx >= n) continue;
        // the claim phase's outcome: a molecule that claimed nothing cannot
        // have won anything; one that claimed knows its direction without a
        // second draw; only first-order firings are drawn again
        const int known = a.dec ? (int)a.dec[idx] : (int)kDecFire;
        if (known == kDecNone) continue;
        const uint32_t v = (uint32_t)a.list.vox[idx];
        const uint32_t id = a.list.ids[idx];
        int32_t i, j, k;
        decode(a.geo, v, i, j, k);
        const BitPos bv = bitpos(a.geo, i, j, k);
        uint32_t u[4] = {0u, 0u, 0u, 0u};
        if (known == kDecFire) philox(id, g, c2, 0u, a.key0, a.key1, u);
        if (GENERAL && known == kDecFire) {
            const ModelDev* M = a.model;
            if (M->n_fo[a.s] > 0 && (uint64_t)u[2] < M->T_fire[a.s]) {
                const ReactionDev R = M->rx[pick_first_order(M, a.s, u[3])];
                if (R.np == 2) {
                    // the neighbour this molecule claimed, if it won it; only
                    // its winner changes the bit of a claimed voxel
                    uint32_t* pb = M->mirror[R.p1];
                    for (int d = 0; d < 12; ++d) {
                        Nb nb;
                        if (!neighbor(a.geo, i, j, k, d, nb)) continue;
                        const BitPos bt = bitpos(a.geo, nb.i, nb.j, nb.k);
                        if (occupied(pb, bt) || !won<HASH>(a, nb, id)) continue;
                        a.occ[v] = (uint16_t)(R.p0 + 1);
                        a.occ[nb.t] = (uint16_t)(R.p1 + 1);
                        bit_set(pb, bt);
                        mark_dirty(dirty, bv.word);
                        mover_leaves(a, idx, v, id, (uint16_t)(R.p0 + 1));
                        const int slot = atomicAdd(&a.sc->births, 1);
                        if (slot < a.births_cap) {
                            Birth b;
                            b.parent = id; b.t = nb.t; b.species = R.p1; b.pad = 0;
                            b.img = img_add(a.list.img[idx], nb.wrap);
                            a.births[slot] = b;
                        } else {
                            atomicOr(&a.sc->err, kErrBirthOverflow);
                        }
                        ++n_r1;
                        break;
                    }
                } else {
                    if (R.np) {
                        a.occ[v] = (uint16_t)(R.p0 + 1);
                    } else {
                        a.occ[v] = 0;
                        bit_clear(a.bits, bv);
                    }
                    mark_dirty(dirty, bv.word);
                    mover_leaves(a, idx, v, id, R.np ? (uint16_t)(R.p0 + 1) : (uint16_t)0);
                    ++n_r1;
                }
                continue;
            }
        }
        const int d = known == kDecFire ? (int)__umulhi(u[0], 12u) : known;
        Nb nb;
        if (!neighbor(a.geo, i, j, k, d, nb)) continue;
        if (!won<HASH>(a, nb, id)) continue;                   // lost, or never claimed
        const BitPos bt = bitpos(a.geo, nb.i, nb.j, nb.k);
        // the bit of a claimed voxel only changes through its winner, so it
        // still tells a vacant target (hop) from a partner (reaction)
        if (!GENERAL || !occupied(a.bits, bt)) {
            bit_move(a.bits, bv, bt);                           // move (Sec. 2.3)
            if (a.live) {
                a.occ[nb.t] = self;
                a.occ[v] = 0;
            }
            a.list.vox[idx] = nb.t;
            if (nb.wrap) a.list.img[idx] = img_add(a.list.img[idx], nb.wrap);
            ++n_hop;
        } else {
            // accepted collision with partner y = o - 1 (Sec. 2.4.2): first
            // product on the partner's voxel, second on the mover's, unless
            // that puts a product outside its compartment (then they trade
            // places).  The partner's voxel is in y's compartment, its bit in
            // y's mirror.
            const ModelDev* M = a.model;
            const int y = (int)a.occ[nb.t] - 1;
            const ReactionDev R = M->rx[M->pair[a.s][y]];
            uint32_t* tb = M->mirror[y];
            const bool straight = R.np == 0 ||
                                  (M->comp[R.p0] == M->comp[y] && (R.np < 2 || M->comp[R.p1] == M->comp[a.s]));
            if (R.np == 0) {
                a.occ[nb.t] = 0;
                bit_clear(tb, bt);
                a.occ[v] = 0;
                bit_clear(a.bits, bv);
            } else if (R.np == 1 && straight) {
                a.occ[nb.t] = (uint16_t)(R.p0 + 1);
                a.occ[v] = 0;
                bit_clear(a.bits, bv);
            } else if (R.np == 1) {
                a.occ[v] = (uint16_t)(R.p0 + 1);
                a.occ[nb.t] = 0;
                bit_clear(tb, bt);
            } else {
                a.occ[nb.t] = (uint16_t)((straight ? R.p0 : R.p1) + 1);
                a.occ[v] = (uint16_t)((straight ? R.p1 : R.p0) + 1);
            }
            mark_dirty(dirty, bt.word);
            mark_dirty(dirty, bv.word);
            mover_leaves(a, idx, v, id, a.occ[v]);
            ++n_r2;
        }
    }
    if (a.collect_stats) {
        flush_stat(&a.sc->stats[kStatHops], n_hop);
        if (GENERAL) {
            flush_stat(&a.sc->stats[kStatReactions2], n_r2);
            flush_stat(&a.sc->stats[kStatReactions1], n_r1);
        }
    }
}

template <bool GENERAL, bool HASH>
__global__ void __launch_bounds__(256) k_commit(const EventArgs a)
{
    commit_body<GENERAL, HASH>(a, event_index(a), blockIdx.x, gridDim.x);
}

void launch_claim(const EventArgs& a, bool general, int blocks, int threads, cudaStream_t st)
{
    const bool hash = a.ct.hash != nullptr;
    if (general) {
        if (hash) k_claim<true, true><<<blocks, threads, 0, st>>>(a);
        else k_claim<true, false><<<blocks, threads, 0, st>>>(a);
    } else {
        if (hash) k_claim<false, true><<<blocks, threads, 0, st>>>(a);
        else k_claim<false, false><<<blocks, threads, 0, st>>>(a);
    }
}

void launch_commit(const EventArgs& a, bool general, int blocks, int threads, cudaStream_t st)
{
    const bool hash = a.ct.hash != nullptr;
    if (general) {
        if (hash) k_commit<true, true><<<blocks, threads, 0, st>>>(a);
        else k_commit<true, false><<<blocks, threads, 0, st>>>(a);
    } else {
        if (hash) k_commit<false, true><<<blocks, threads, 0, st>>>(a);
        else k_commit<false, false><<<blocks, threads, 0, st>>>(a);
    }
}

// ---------------------------------------------------------------------------
// persistent stretch of events of one species without reactions
//
// One cooperative launch sized to the SMs (see kRunShapes).  Thread x owns the
// molecules x, x + T, x + 2T, ... (T threads in all) of the list for the whole
// stretch and keeps their voxel, id and claim state in registers; each event
// is claim phase -> grid barrier -> commit phase -> grid barrier.  A claimant
// remembers the slot that holds its voxel's claim, so the commit phase reads
// that one slot, and the next event's claim phase empties it again (the
// tables alternate, so the table being emptied is not in use).
// ---------------------------------------------------------------------------
constexpr unsigned int kBarrierMaxSpins = 1u << 28;
constexpr int kGroup = 1;                                  // molecules in flight per thread

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier: block 0 adds 2^31 - (blocks - 1), every other block adds 1,
// so the top bit of the arrival word flips exactly when all have arrived.
// The wait is bounded by timeout_ns of wall time (one second unless the
// caller sets it) and by a spin count: on time-out the block raises
// kErrBarrierTimeout and every thread of it returns false.  `phantom` counts
// arrivals awaited from blocks that do not exist (0 outside tests): with
// phantom > 0 the bit never flips and every block waits out its bound.
__device__ __forceinline__ bool grid_barrier(BarrierState* bs, int32_t* err, uint64_t timeout_ns,
                                             uint32_t phantom)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int inc = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u + phantom) : 1u;
        __threadfence();
        const unsigned int old = atomicAdd(&bs->arrive, inc);
        volatile unsigned int* word = &bs->arrive;
        int good = 1;
        uint64_t t0 = 0;
        for (unsigned int spins = 0; ((old ^ *word) & 0x80000000u) == 0u; ++spins) {
            if ((spins & 1023u) == 0u) {
                const uint64_t now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                // the spin count bounds the wait even if the timer were to stall
                if (now - t0 > timeout_ns || spins >= kBarrierMaxSpins) {
                    atomicOr(err, kErrBarrierTimeout);
                    good = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// packed claim state of one molecule: bit 31 claimed, bits 27-30 direction,
// bits 0-26 slot (hash tables of at most 2^27 slots).  A thread that leaves
// through a failed barrier leaves the others to fail theirs within the same
// bound; the host sees kErrBarrierTimeout.
constexpr uint32_t kClaimed = 0x80000000u;

template <bool HASH, int M, int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_hop_run(const RunArgs r)
{
    // per-molecule state lives in shared memory, [m][thread] (conflict-free)
    extern __shared__ uint32_t sm_state[];
    uint32_t* s_vox = sm_state;
    uint32_t* s_ids = sm_state + M * THREADS;
    uint32_t* s_st = sm_state + 2 * M * THREADS;
    const EventArgs& a = r.ev;
    const int32_t n = *a.count;
    const int T = gridDim.x * THREADS;
    const int gt = blockIdx.x * THREADS + threadIdx.x;
    const uint32_t c2 = ((uint32_t)a.s << 4) | kTagEvent;
    const uint16_t self = (uint16_t)(a.s + 1);
    int mine = 0;                                   // molecules of this thread
    for (int m = 0; m < M; ++m) {
        const int idx = gt + m * T;
        if (idx < n) {
            s_vox[m * THREADS + threadIdx.x] = (uint32_t)a.list.vox[idx];
            s_ids[m * THREADS + threadIdx.x] = a.list.ids[idx];
            mine = m + 1;
        }
        s_st[m * THREADS + threadIdx.x] = 0u;
    }
    unsigned long long n_hop = 0;
    for (int e = 0; e < r.n_events; ++e) {
        const uint32_t g = a.g + (uint32_t)e;
        uint64_t* tab = r.tables[g & 1u];
        uint64_t* old = r.tables[(g & 1u) ^ 1u];
        // ---- claim phase: kGroup molecules at a time, their loads and first
        // claim attempts in flight together ----
        for (int m0 = 0; m0 < mine; m0 += kGroup) {
            Nb nb[kGroup];
            BitPos bp[kGroup];
            uint32_t idg[kGroup], stg[kGroup], home[kGroup], word[kGroup];
            uint64_t hv[kGroup], prev[kGroup];
            bool ok[kGroup], tried[kGroup];
#pragma unroll
            for (int x = 0; x < kGroup; ++x) {
                const int m = m0 + x;
                ok[x] = false;
                tried[x] = false;
                stg[x] = 0u;
                idg[x] = 0u;
                home[x] = 0u;
                if (m >= mine) continue;
                const int q = m * THREADS + threadIdx.x;
                const uint32_t before = s_st[q];
                if (HASH && (before & kClaimed)) old[before & 0x07FFFFFFu] = kEmptySlot;   // previous event
                idg[x] = s_ids[q];
                int32_t i, j, k;
                decode(a.geo, s_vox[q], i, j, k);
                uint32_t u[4];
                philox(idg[x], g, c2, 0u, a.key0, a.key1, u);
                const int d = (int)__umulhi(u[0], 12u);
                stg[x] = (uint32_t)d << 27;
                ok[x] = neighbor(a.geo, i, j, k, d, nb[x]);
                if (ok[x]) {
                    bp[x] = bitpos(a.geo, nb[x].i, nb[x].j, nb[x].k);
                    if (HASH) home[x] = slot_of(a.geo, (uint32_t)nb[x].t, nb[x].i, nb[x].j, nb[x].k, a.ct.hash_bits);
                }
            }
#pragma unroll
            for (int x = 0; x < kGroup; ++x) {
                if (!ok[x]) continue;
                word[x] = __ldcg(&a.bits[bp[x].word]);
                if (HASH) hv[x] = __ldcg((const unsigned long long*)&tab[home[x]]);
            }
#pragma unroll
            for (int x = 0; x < kGroup; ++x) {
                ok[x] = ok[x] && !(word[x] & bp[x].mask);            // vacant target
                if (!ok[x]) continue;
                if (HASH) {
                    if (hv[x] == kEmptySlot) {
                        prev[x] = atomicCAS((unsigned long long*)&tab[home[x]], (unsigned long long)kEmptySlot,
                                            (unsigned long long)(((uint64_t)nb[x].t << 32) | idg[x]));
                        tried[x] = true;
                    }
                } else {
                    atomicMin(&a.ct.direct[nb[x].t], idg[x]);
                    stg[x] |= kClaimed;
                }
            }
            if (HASH) {
#pragma unroll
                for (int x = 0; x < kGroup; ++x) {
                    if (!ok[x]) continue;
                    int32_t slot;
                    if (tried[x] && prev[x] == kEmptySlot) slot = (int32_t)home[x];
                    else slot = hash_claim_from(tab, a.ct.hash_bits, (uint32_t)nb[x].t, idg[x], home[x],
                                                tried[x] ? prev[x] : hv[x], &a.sc->err);
                    if (slot >= 0) stg[x] |= kClaimed | (uint32_t)slot;
                }
            }
#pragma unroll
            for (int x = 0; x < kGroup; ++x)
                if (m0 + x < mine) s_st[(m0 + x) * THREADS + threadIdx.x] = stg[x];
        }
        if (!grid_barrier(r.barrier, &a.sc->err, r.barrier_timeout_ns, r.barrier_phantom)) return;
        // ---- commit phase: slot reads of a group in flight together ----
        for (int m0 = 0; m0 < mine; m0 += kGroup) {
            uint32_t stg[kGroup], cw[kGroup];
            uint64_t tv[kGroup];
            Nb nb[kGroup];
            int32_t ci[kGroup], cj[kGroup], ck[kGroup];
#pragma unroll
            for (int x = 0; x < kGroup; ++x) {
                stg[x] = (m0 + x < mine) ? s_st[(m0 + x) * THREADS + threadIdx.x] : 0u;
                if (HASH && (stg[x] & kClaimed)) tv[x] = __ldcg((const unsigned long long*)&tab[stg[x] & 0x07FFFFFFu]);
            }
#pragma unroll
            for (int x = 0; x < kGroup; ++x) {
                if (!(stg[x] & kClaimed)) continue;
                decode(a.geo, s_vox[(m0 + x) * THREADS + threadIdx.x], ci[x], cj[x], ck[x]);
                neighbor(a.geo, ci[x], cj[x], ck[x], (int)((stg[x] >> 27) & 15u), nb[x]);
                if (!HASH) cw[x] = __ldcg(&a.ct.direct[nb[x].t]);
            }
#pragma unroll
            for (int x = 0; x < kGroup; ++x) {
                if (!(stg[x] & kClaimed)) continue;
                const int q = (m0 + x) * THREADS + threadIdx.x;
                const uint32_t id = s_ids[q];
                bool win;
                if (HASH) {
                    win = (uint32_t)tv[x] == id;
                } else {
                    win = cw[x] == id;
                    if (win) a.ct.direct[nb[x].t] = kNoClaim;
                }
                if (!win) continue;
                const uint32_t v = s_vox[q];
                bit_move(a.bits, bitpos(a.geo, ci[x], cj[x], ck[x]), bitpos(a.geo, nb[x].i, nb[x].j, nb[x].k));
                if (a.live) {
                    a.occ[nb[x].t] = self;
                    a.occ[v] = 0;
                }
                if (nb[x].wrap) {
                    const int idx = gt + (m0 + x) * T;
                    a.list.img[idx] = img_add(a.list.img[idx], nb[x].wrap);
                }
                s_vox[q] = (uint32_t)nb[x].t;
                ++n_hop;
            }
        }
        if (!grid_barrier(r.barrier, &a.sc->err, r.barrier_timeout_ns, r.barrier_phantom)) return;
    }
    // leave both tables empty: the last event's slots (the one before was
    // emptied during the last claim phase)
    if (HASH && r.n_events > 0) {
        uint64_t* last = r.tables[(a.g + (uint32_t)r.n_events - 1u) & 1u];
        for (int m = 0; m < mine; ++m) {
            const uint32_t stq = s_st[m * THREADS + threadIdx.x];
            if (stq & kClaimed) last[stq & 0x07FFFFFFu] = kEmptySlot;
        }
    }
    for (int m = 0; m < mine; ++m) a.list.vox[gt + m * T] = (int32_t)s_vox[m * THREADS + threadIdx.x];
    if (a.collect_stats) {
        flush_stat(&a.sc->stats[kStatHops], n_hop);
        flush_stat(&a.sc->stats[kStatAttempts], (unsigned long long)mine * (unsigned long long)r.n_events);
    }
}

// Launch shapes: two 768-thread blocks per SM (<= 42 registers) with up to 6
// molecules per thread, or one 768-thread block per SM with up to 16
// (3 x 16 x 768 words = 144 KB of shared memory).  More resident threads
// beat more molecules in flight per thread here (measured: the kernel is
// bound by L2 operations, not by per-thread latency chains).  With 16
// molecules per thread it only matches one claim and one commit launch per
// event, and with 24 it took 1.85 times as long (2.2M molecules at 512^3),
// so larger species take the per-event launches (or the tile kernel).
struct RunShape {
    int per_thread, threads, blocks_per_sm;
};
static const RunShape kRunShapes[] = {
    {2, 768, 2}, {4, 768, 2}, {6, 768, 2}, {8, 768, 1}, {12, 768, 1}, {16, 768, 1}};

int run_capacity(int64_t n, int* threads_per_block, int* blocks, int sm_count, int min_per_thread)
{
    for (const RunShape& sh : kRunShapes) {
        const int64_t T = (int64_t)sh.threads * sh.blocks_per_sm * sm_count;
        if (sh.per_thread >= min_per_thread && n <= (int64_t)sh.per_thread * T) {
            *threads_per_block = sh.threads;
            *blocks = sh.blocks_per_sm * sm_count;
            return sh.per_thread;
        }
    }
    return 0;
}

template <bool HASH, int M, int THREADS, int MINB>
static cudaError_t launch_run_t(const RunArgs& r, int blocks, int threads, cudaStream_t st)
{
    if (threads != THREADS) return cudaErrorInvalidValue;
    const size_t smem = (size_t)3 * M * THREADS * sizeof(uint32_t);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute((const void*)k_hop_run<HASH, M, THREADS, MINB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    void* args[] = {const_cast<RunArgs*>(&r)};
    return cudaLaunchCooperativeKernel((const void*)k_hop_run<HASH, M, THREADS, MINB>, dim3(blocks), dim3(threads),
                                       args, smem, st);
}

template <bool HASH>
static cudaError_t launch_run_h(const RunArgs& r, int blocks, int threads, int per_thread, cudaStream_t st)
{
    switch (per_thread) {
    case 2: return launch_run_t<HASH, 2, 768, 2>(r, blocks, threads, st);
    case 4: return launch_run_t<HASH, 4, 768, 2>(r, blocks, threads, st);
    case 6: return launch_run_t<HASH, 6, 768, 2>(r, blocks, threads, st);
    case 8: return launch_run_t<HASH, 8, 768, 1>(r, blocks, threads, st);
    case 12: return launch_run_t<HASH, 12, 768, 1>(r, blocks, threads, st);
    case 16: return launch_run_t<HASH, 16, 768, 1>(r, blocks, threads, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_run(const RunArgs& r, int blocks, int threads, int per_thread, cudaStream_t st)
{
    return r.ev.ct.hash ? launch_run_h<true>(r, blocks, threads, per_thread, st)
                        : launch_run_h<false>(r, blocks, threads, per_thread, st);
}

// ---------------------------------------------------------------------------
// reconcile: bring the list of species x in line with the grid after an event
// with reactions.  An entry whose voxel holds x stays; one whose voxel holds
// species y (a product that inherited this molecule's identity) moves to y's
// list; one whose voxel is empty is dropped.  Species with reactions always
// keep their codes in occ, and a vacant voxel never keeps the code of one, so
// "occupied and code y + 1" identifies y exactly.  Only entries in bricks the
// commit marked (a voxel there changed species) can have changed: the others
// stay where they are without a look at the grid.  The entries that leave are
// marked (voxel -1) and their slots noted; the fill pass then moves the
// survivors from the end of the list into the slots below the new length.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_alloc(int* counter, bool want)
{
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, want);
    if (!mask) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return want ? base + __popc(mask & ((1u << lane) - 1u)) : -1;
}

// The slots of the lists' leavers share the scratch arrays: list x's take the
// range after those of the lists in `before` (the due species' own first,
// then the partner lists in their order), so the lists fill side by side.
__device__ __forceinline__ int32_t leave_base(const Scalars* sc, uint32_t before)
{
    int32_t base = 0;
    for (uint32_t m = before; m; m &= m - 1u) base += sc->tmp_count[__ffs(m) - 1];
    return base;
}

__device__ __forceinline__ void reconcile_body(const ReconcileArgs& r, uint32_t g, int blk, int nblk,
                                               uint32_t before)
{
    const int32_t n = r.sc->counts[r.x];
    const uint16_t self = (uint16_t)(r.x + 1);
    const uint32_t* dirty = r.dirty[g & 1u];
    int32_t* leave = r.tmp.vox + leave_base(r.sc, before);   // slots of the entries that leave
    const int stride = nblk * blockDim.x;
    for (int base = blk * blockDim.x; base < n; base += stride) {
        const int idx = base + threadIdx.x;
        int32_t v = 0;
        uint16_t o = 0;
        bool leaving = false;
        if (idx < n) {
            v = r.list.vox[idx];
            int32_t i, j, k;
            decode(r.geo, (uint32_t)v, i, j, k);
            const BitPos bp = bitpos(r.geo, i, j, k);
            if ((dirty[bp.word >> 5] >> (bp.word & 31u)) & 1u) {
                o = occupied(r.bits, bp) ? r.occ[v] : (uint16_t)0;
                leaving = o != self;
            }
        }
        const int slot = warp_alloc(&r.sc->tmp_count[r.x], leaving);
        if (!leaving) continue;
        leave[slot] = idx;
        const uint32_t id = r.list.ids[idx];
        const uint64_t img = r.list.img[idx];
        r.list.vox[idx] = -1;
        if (o != 0 && o != kBlocked) {
            const int y = o - 1;
            const SpeciesList dst = r.model->lists[y];
            const int s2 = atomicAdd(&r.sc->counts[y], 1);
            if (s2 < dst.cap) {
                dst.vox[s2] = v;
                dst.ids[s2] = id;
                dst.img[s2] = img;
            } else {
                atomicOr(&r.sc->err, kErrListOverflow);
            }
        }
    }
}

__device__ __forceinline__ uint32_t reconcile_event(const ReconcileArgs& r)
{
    return r.g_base ? __ldcg(r.g_base) + r.g : r.g;
}

__global__ void __launch_bounds__(256) k_reconcile(const ReconcileArgs r, uint32_t before)
{
    reconcile_body(r, reconcile_event(r), blockIdx.x, gridDim.x, before);
}

// The fill of fill_body for the block whose threads (and atomics) wrote the
// list's entries and counts in the same launch: counts and entries are read
// through L2.
__device__ __forceinline__ void fill_list(const SpeciesList& list, int32_t* count, int32_t k_left,
                                          const int32_t* leave, int32_t* holes, int32_t* surv, int32_t* err)
{
    __shared__ int s_h, s_s;
    const int32_t n = __ldcg(count);
    const int32_t k = min(k_left, n);
    if (k <= 0) return;
    const int32_t n2 = n - k;
    if (threadIdx.x == 0) {
        s_h = 0;
        s_s = 0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
        const int32_t h = __ldcg(leave + q);
        if (h < n2) holes[atomicAdd(&s_h, 1)] = h;
    }
    for (int p = n2 + threadIdx.x; p < n; p += blockDim.x)
        if (__ldcg(list.vox + p) >= 0) surv[atomicAdd(&s_s, 1)] = p;
    __syncthreads();
    const int m = min(s_h, s_s);
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
        const int32_t h = holes[q], p = surv[q];
        list.vox[h] = __ldcg(list.vox + p);
        list.ids[h] = __ldcg(list.ids + p);
        list.img[h] = __ldcg(list.img + p);
    }
    if (threadIdx.x == 0) {
        *count = n2;
        if (s_h != s_s) atomicOr(err, kErrListOverflow);
    }
}

// One block per list: k entries left; the new length is n - k.  Every slot
// below it that an entry left (a hole) takes one of the surviving entries at
// or above it (there are as many); entries that left above it are simply cut
// off.  The list's holes and survivors go to its range of the scratch arrays.
// (fill_list does the same inside the launch that wrote the entries.)
__device__ __forceinline__ void fill_body(const ReconcileArgs& r, uint32_t before)
{
    __shared__ int s_h, s_s;
    const int32_t n = r.sc->counts[r.x];
    const int32_t k = min(r.sc->tmp_count[r.x], n);
    if (k <= 0) return;
    const int32_t n2 = n - k;
    const int32_t base = leave_base(r.sc, before);
    const int32_t* leave = r.tmp.vox + base;
    int32_t* holes = reinterpret_cast<int32_t*>(r.tmp.ids) + base;
    int32_t* surv = reinterpret_cast<int32_t*>(r.tmp.img) + base;
    if (threadIdx.x == 0) {
        s_h = 0;
        s_s = 0;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
        const int32_t h = leave[q];
        if (h < n2) holes[atomicAdd(&s_h, 1)] = h;
    }
    for (int p = n2 + threadIdx.x; p < n; p += blockDim.x)
        if (r.list.vox[p] >= 0) surv[atomicAdd(&s_s, 1)] = p;
    __syncthreads();
    const int m = min(s_h, s_s);
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
        const int32_t h = holes[q], p = surv[q];
        r.list.vox[h] = r.list.vox[p];
        r.list.ids[h] = r.list.ids[p];
        r.list.img[h] = r.list.img[p];
    }
    if (threadIdx.x == 0) {
        r.sc->counts[r.x] = n2;
        if (s_h != s_s) atomicOr(&r.sc->err, kErrListOverflow);
    }
}

// block q fills list f.x[q]; block 0 advances the event index when asked
// (no block of this launch reads it otherwise)
__global__ void __launch_bounds__(1024) k_fill(const ListFill f)
{
    ReconcileArgs r = f.r;
    r.x = f.x[blockIdx.x];
    r.list = f.list[blockIdx.x];
    fill_body(r, f.before[blockIdx.x]);
    if (blockIdx.x == 0 && threadIdx.x == 0 && r.g_bump) *r.g_bump = reconcile_event(r) + 1u;
}

void launch_reconcile(const ReconcileArgs& r, uint32_t before, int blocks, int threads, cudaStream_t st)
{
    k_reconcile<<<blocks, threads, 0, st>>>(r, before);
}

void launch_fill(const ListFill& f, cudaStream_t st)
{
    k_fill<<<f.n, 1024, 0, st>>>(f);
}

// A whole event of a short list of a species with reactions in one block:
// the claim phase, a block barrier (after which every claim of the event is
// in place and visible to the block), the commit phase, another barrier, and
// the fill of the species' own list (its leavers' slots come first in the
// scratch arrays).  Claims the block reads back and bits it tests change only
// through their winner, as across launches.
template <bool HASH>
__global__ void __launch_bounds__(kEventOneThreads) k_event_one(const EventArgs a)
{
    const uint32_t g = event_index(a);
    claim_body<true, HASH>(a, g, 0, 1);
    __syncthreads();
    commit_body<true, HASH>(a, g, 0, 1);
    __syncthreads();
    fill_list(a.list, &a.sc->counts[a.s], __ldcg(&a.sc->tmp_count[a.s]), a.leave, a.holes, a.surv, &a.sc->err);
    if (threadIdx.x == 0 && a.g_bump) *a.g_bump = g + 1u;
}

void launch_event_one(const EventArgs& a, cudaStream_t st)
{
    if (a.ct.hash) k_event_one<true><<<1, kEventOneThreads, 0, st>>>(a);
    else k_event_one<false><<<1, kEventOneThreads, 0, st>>>(a);
}

// ---------------------------------------------------------------------------
// births: one block sorts the births of this event by parent id (bitonic, in
// shared memory) and hands out ids next_id, next_id + 1, ... in that order.
// ---------------------------------------------------------------------------
constexpr int kBirthSortMax = 8192;

__device__ __forceinline__ void births_body(const EventArgs& a)
{
    extern __shared__ unsigned long long keys[];
    int nb = a.sc->births;
    if (nb == 0) return;
    if (nb > a.births_cap || nb > kBirthSortMax) {
        if (threadIdx.x == 0) atomicOr(&a.sc->err, kErrBirthOverflow);
        nb = min(min(nb, a.births_cap), kBirthSortMax);
    }
    int np2 = 1;
    while (np2 < nb) np2 <<= 1;
    for (int x = threadIdx.x; x < np2; x += blockDim.x)
        keys[x] = x < nb ? (((unsigned long long)a.births[x].parent << 32) | (unsigned)x) : ~0ull;
    __syncthreads();
    for (int size = 2; size <= np2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int x = threadIdx.x; x < np2; x += blockDim.x) {
                const int y = x ^ stride;
                if (y > x) {
                    const bool up = (x & size) == 0;
                    const unsigned long long kx = keys[x], ky = keys[y];
                    if ((kx > ky) == up) { keys[x] = ky; keys[y] = kx; }
                }
            }
            __syncthreads();
        }
    }
    const uint32_t base_id = a.sc->next_id;
    for (int x = threadIdx.x; x < nb; x += blockDim.x) {
        const Birth b = a.births[(int)(keys[x] & 0xFFFFFFFFu)];
        const SpeciesList dst = a.model->lists[b.species];
        const int slot = atomicAdd(&a.sc->counts[b.species], 1);
        if (slot < dst.cap) {
            dst.vox[slot] = b.t;
            dst.ids[slot] = base_id + (uint32_t)x;
            dst.img[slot] = b.img;
        } else {
            atomicOr(&a.sc->err, kErrListOverflow);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.sc->next_id = base_id + (uint32_t)nb;
        if (a.collect_stats) a.sc->stats[kStatBirths] += (unsigned long long)nb;
        a.sc->births = 0;
    }
}

__global__ void __launch_bounds__(1024) k_births(const EventArgs a)
{
    births_body(a);
    if (threadIdx.x == 0 && a.g_bump) *a.g_bump = event_index(a) + 1u;
}

void launch_births(const EventArgs& a, cudaStream_t st)
{
    static bool configured = false;
    const int smem = kBirthSortMax * (int)sizeof(unsigned long long);
    if (!configured) {
        cudaFuncSetAttribute(k_births, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        configured = true;
    }
    k_births<<<1, 1024, smem, st>>>(a);
}

// ---------------------------------------------------------------------------
// populate and list maintenance
// ---------------------------------------------------------------------------
__global__ void k_fill_u32(uint32_t* p, uint32_t value, size_t n)
{
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x)
        p[x] = value;
}

void launch_fill_u32(uint32_t* p, uint32_t value, size_t n, int blocks, cudaStream_t st)
{
    k_fill_u32<<<blocks, 256, 0, st>>>(p, value, n);
}

__global__ void k_fill_u64(uint64_t* p, uint64_t value, size_t n)
{
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < n; x += (size_t)gridDim.x * blockDim.x)
        p[x] = value;
}

void launch_fill_u64(uint64_t* p, uint64_t value, size_t n, int blocks, cudaStream_t st)
{
    k_fill_u64<<<blocks, 256, 0, st>>>(p, value, n);
}

// exact species grid for read-out: the codes of species with reactions where
// the mirrors say occupied, zero elsewhere; species without reactions are
// written afterwards from their lists (they do not keep codes while moving).
// A voxel is occupied when its bit is set in every compartment's mirror (in
// all but its own compartment's it is a wall).
__global__ void k_materialize(uint16_t* out, const uint16_t* occ, const uint32_t* bits0, uint64_t words,
                              int n_mirrors, Geometry G, int64_t V)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t i, j, k;
        decode(G, (uint32_t)v, i, j, k);
        const BitPos b = bitpos(G, i, j, k);
        bool full = true;
        for (int c = 0; c < n_mirrors; ++c) full = full && occupied(bits0 + (uint64_t)c * words, b);
        out[v] = full ? occ[v] : (uint16_t)0;
    }
}

void launch_materialize(uint16_t* out, const uint16_t* occ, const uint32_t* bits0, uint64_t words,
                        int n_mirrors, const Geometry& geo, int64_t V, int blocks, cudaStream_t st)
{
    k_materialize<<<blocks, 256, 0, st>>>(out, occ, bits0, words, n_mirrors, geo, V);
}

// walls: one thread per mirror word builds that word of every mirror from
// the labels of its 4 x 4 x 2 brick (voxels outside the lattice stay clear)
__global__ void k_mirror_walls(uint32_t* bits0, uint64_t words, int n, const uint8_t* labels, Geometry G)
{
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words;
         w += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t bi = (uint32_t)(w % G.nbi);
        const uint32_t bj = (uint32_t)((w / G.nbi) % G.nbj);
        const uint32_t bk = (uint32_t)(w / ((uint64_t)G.nbi * G.nbj));
        uint32_t m[kMaxCompartments];
        for (int c = 0; c < n; ++c) m[c] = 0u;
        for (uint32_t b = 0; b < 32; ++b) {
            const int32_t i = (int32_t)(bi * 4 + (b & 3u));
            const int32_t j = (int32_t)(bj * 4 + ((b >> 2) & 3u));
            const int32_t k = (int32_t)(bk * 2 + (b >> 4));
            if (i >= G.ni || j >= G.nj || k >= G.nk) continue;
            const int lab = labels[(uint64_t)i + (uint64_t)G.ni * ((uint64_t)j + (uint64_t)G.nj * (uint64_t)k)];
            for (int c = 0; c < n; ++c)
                if (c != lab) m[c] |= 1u << b;
        }
        for (int c = 0; c < n; ++c) bits0[(uint64_t)c * words + w] = m[c];
    }
}

void launch_mirror_walls(uint32_t* bits0, uint64_t words, int n, const uint8_t* labels, const Geometry& geo,
                         int blocks, cudaStream_t st)
{
    k_mirror_walls<<<blocks, 256, 0, st>>>(bits0, words, n, labels, geo);
}

__global__ void k_label_keys(const uint32_t* vals, const uint8_t* labels, uint32_t* keys, int64_t n)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        keys[r] = labels[vals[r]];
}

void launch_label_keys(const uint32_t* vals, const uint8_t* labels, uint32_t* keys, int64_t n, int blocks,
                       cudaStream_t st)
{
    k_label_keys<<<blocks, 256, 0, st>>>(vals, labels, keys, n);
}

__global__ void k_scatter_codes(uint16_t* out, const SpeciesList L, const int32_t* count, uint16_t code)
{
    const int32_t n = *count;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        out[L.vox[x]] = code;
}

void launch_scatter_codes(uint16_t* out, const SpeciesList& list, const int32_t* count, uint16_t code,
                          int blocks, cudaStream_t st)
{
    k_scatter_codes<<<blocks, 256, 0, st>>>(out, list, count, code);
}

// Placement by selection.  The key of voxel v is word 0 of Philox(seed; v, 0,
// 1, 0); the species take the first voxels of each compartment in (key,
// voxel) order, so only the voxels whose key lies in
// the bins that cover them need sorting.  Pass 1 histograms the top
// kPlaceBits bits of every voxel's key per compartment; pass 2 keeps the
// voxels up to each compartment's last needed bin.
__global__ void k_place_hist(uint32_t V, uint32_t key0, uint32_t key1, const uint8_t* labels, int nc,
                             uint32_t* hist)
{
    extern __shared__ uint32_t s_bins[];
    const int nb = nc << kPlaceBits;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s_bins[b] = 0u;
    __syncthreads();
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        uint32_t u[4];
        philox(v, 0u, kTagPopulate, 0u, key0, key1, u);
        const int c = labels ? (int)labels[v] : 0;
        atomicAdd(&s_bins[(c << kPlaceBits) | (int)(u[0] >> (32 - kPlaceBits))], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        if (s_bins[b]) atomicAdd(&hist[b], s_bins[b]);
}

void launch_place_hist(uint32_t V, uint32_t key0, uint32_t key1, const uint8_t* labels, int nc, uint32_t* hist,
                       int blocks, cudaStream_t st)
{
    const int smem = (nc << kPlaceBits) * (int)sizeof(uint32_t);
    static int configured = 48 * 1024;
    if (smem > configured) {
        cudaFuncSetAttribute(k_place_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        configured = smem;
    }
    k_place_hist<<<blocks, 256, smem, st>>>(V, key0, key1, labels, nc, hist);
}

__global__ void k_place_pick(uint32_t V, uint32_t key0, uint32_t key1, const uint8_t* labels, PlaceLimits lim,
                             uint32_t* out_vox, uint32_t* out_key, int32_t* count, int32_t cap, int32_t* err)
{
    for (uint32_t v0 = blockIdx.x * blockDim.x; v0 < V; v0 += gridDim.x * blockDim.x) {   // whole warps
        const uint32_t v = v0 + threadIdx.x;
        bool want = false;
        uint32_t key = 0u;
        if (v < V) {
            uint32_t u[4];
            philox(v, 0u, kTagPopulate, 0u, key0, key1, u);
            key = u[0];
            want = (int)(key >> (32 - kPlaceBits)) <= lim.bin[labels ? (int)labels[v] : 0];
        }
        const int slot = warp_alloc(count, want);
        if (want) {
            if (slot < cap) {
                out_vox[slot] = v;
                out_key[slot] = key;
            } else {
                atomicOr(err, kErrListOverflow);
            }
        }
    }
}

void launch_place_pick(uint32_t V, uint32_t key0, uint32_t key1, const uint8_t* labels, const PlaceLimits& lim,
                       uint32_t* out_vox, uint32_t* out_key, int32_t* count, int32_t cap, int32_t* err, int blocks,
                       cudaStream_t st)
{
    k_place_pick<<<blocks, 256, 0, st>>>(V, key0, key1, labels, lim, out_vox, out_key, count, cap, err);
}

struct Offsets {
    int64_t off[kMaxSpecies + 1];
};

// molecule r (id r) belongs to the species whose id range holds r and takes
// that species' next voxel of the sorted order
__global__ void k_populate_scatter(const uint32_t* sorted_vox, int64_t n_total, Offsets o, Offsets start,
                                   int n_species, uint16_t* occ, Geometry G, const ModelDev* model)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_total;
         r += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
        while (s + 1 < n_species && r >= o.off[s + 1]) ++s;
        const int64_t a = r - o.off[s];
        const uint32_t v = sorted_vox[start.off[s] + a];
        occ[v] = (uint16_t)(s + 1);
        int32_t i, j, k;
        decode(G, v, i, j, k);
        bit_set(model->mirror[s], bitpos(G, i, j, k));
        const SpeciesList L = model->lists[s];
        L.vox[a] = (int32_t)v;
        L.ids[a] = (uint32_t)r;
        L.img[a] = 0ull;
    }
}

void launch_populate_scatter(const uint32_t* sorted_vox, int64_t n_total, const int64_t* offsets,
                             const int64_t* starts, int n_species, uint16_t* occ, const Geometry& geo,
                             const ModelDev* model, int blocks, cudaStream_t st)
{
    Offsets o, b;
    for (int s = 0; s <= kMaxSpecies; ++s) {
        o.off[s] = s <= n_species ? offsets[s] : offsets[n_species];
        b.off[s] = s < n_species ? starts[s] : 0;
    }
    k_populate_scatter<<<blocks, 256, 0, st>>>(sorted_vox, n_total, o, b, n_species, occ, geo, model);
}

// Morton (Z-order) key of the voxel of each list entry (compact code)
__global__ void k_morton_keys(const SpeciesList L, const int32_t* count, int32_t limit, Geometry G, uint32_t* keys,
                              uint32_t* vals)
{
    const int32_t n = min(*count, limit);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        int32_t i, j, k;
        decode(G, (uint32_t)L.vox[idx], i, j, k);
        keys[idx] = morton(G, i, j, k);
        vals[idx] = (uint32_t)idx;
    }
}

void launch_morton_keys(const SpeciesList& list, const int32_t* count, int32_t limit, const Geometry& geo,
                        uint32_t* keys, uint32_t* vals, int blocks, cudaStream_t st)
{
    k_morton_keys<<<blocks, 256, 0, st>>>(list, count, limit, geo, keys, vals);
}

uint32_t morton_sort_bits(const Geometry& geo) { return geo.mort_bits; }

__global__ void k_permute(const SpeciesList src, const SpeciesList dst, const uint32_t* perm, const int32_t* count,
                          int32_t limit)
{
    const int32_t n = min(*count, limit);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const uint32_t p = perm[r];
        dst.vox[r] = src.vox[p];
        dst.ids[r] = src.ids[p];
        dst.img[r] = src.img[p];
    }
}

void launch_permute(const SpeciesList& src, const SpeciesList& dst, const uint32_t* perm,
                    const int32_t* count, int32_t limit, int blocks, cudaStream_t st)
{
    k_permute<<<blocks, 256, 0, st>>>(src, dst, perm, count, limit);
}

__global__ void k_copy_list(const SpeciesList src, const SpeciesList dst, const int32_t* count, int32_t limit)
{
    const int32_t n = min(*count, limit);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        dst.vox[r] = src.vox[r];
        dst.ids[r] = src.ids[r];
        dst.img[r] = src.img[r];
    }
}

void launch_copy_list(const SpeciesList& src, const SpeciesList& dst, const int32_t* count, int32_t limit,
                      int blocks, cudaStream_t st)
{
    k_copy_list<<<blocks, 256, 0, st>>>(src, dst, count, limit);
}

__global__ void k_mirror_from_list(uint32_t* bits, Geometry G, const SpeciesList L, const int32_t* count)
{
    const int32_t n = *count;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        int32_t i, j, k;
        decode(G, (uint32_t)L.vox[x], i, j, k);
        bit_set(bits, bitpos(G, i, j, k));
    }
}

void launch_mirror_from_list(uint32_t* bits, const Geometry& geo, const SpeciesList& list, const int32_t* count,
                             int blocks, cudaStream_t st)
{
    k_mirror_from_list<<<blocks, 256, 0, st>>>(bits, geo, list, count);
}

__global__ void k_mirror_from_list_checked(uint32_t* bits, Geometry G, const SpeciesList L, const int32_t* count,
                                           int64_t V, int32_t* err)
{
    const int32_t n = *count;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const int32_t v = L.vox[x];
        if (v < 0 || (int64_t)v >= V || L.ids[x] == kNoClaim) {
            atomicOr(err, kErrBadInput);
            continue;
        }
        int32_t i, j, k;
        decode(G, (uint32_t)v, i, j, k);
        const BitPos b = bitpos(G, i, j, k);
        if (atomicOr(&bits[b.word], b.mask) & b.mask) atomicOr(err, kErrBadInput);   // a second molecule here
    }
}

void launch_mirror_from_list_checked(uint32_t* bits, const Geometry& geo, const SpeciesList& list,
                                     const int32_t* count, int64_t V, int32_t* err, int blocks, cudaStream_t st)
{
    k_mirror_from_list_checked<<<blocks, 256, 0, st>>>(bits, geo, list, count, V, err);
}

// ---------------------------------------------------------------------------
// batched launches: every active replica runs its own next event (or list
// pass) inside one launch; block b belongs to the item whose block range
// holds it.  Replicas in a batch use per-voxel claim words.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_find(const BatchLaunch& bl, int b, int* nblk)
{
    int lo = 0, hi = bl.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bl.item[mid].block0 <= b) lo = mid;
        else hi = mid - 1;
    }
    *nblk = (lo + 1 < bl.n ? bl.item[lo + 1].block0 : bl.total_blocks) - bl.item[lo].block0;
    return lo;
}

__global__ void __launch_bounds__(256) k_claim_batch(const EventArgs* tmpl, const BatchLaunch bl)
{
    int nblk;
    const BatchItem I = bl.item[batch_find(bl, blockIdx.x, &nblk)];
    const EventArgs a = tmpl[I.rep * kMaxSpecies + I.sel];
    claim_body<true, false>(a, I.g, blockIdx.x - I.block0, nblk);
}

__global__ void __launch_bounds__(256) k_commit_batch(const EventArgs* tmpl, const BatchLaunch bl)
{
    int nblk;
    const BatchItem I = bl.item[batch_find(bl, blockIdx.x, &nblk)];
    const EventArgs a = tmpl[I.rep * kMaxSpecies + I.sel];
    commit_body<true, false>(a, I.g, blockIdx.x - I.block0, nblk);
}

__global__ void __launch_bounds__(256) k_reconcile_batch(const ReconcileArgs* tmpl, const BatchLaunch bl)
{
    int nblk;
    const BatchItem I = bl.item[batch_find(bl, blockIdx.x, &nblk)];
    const ReconcileArgs r = tmpl[I.rep * kMaxSpecies + I.sel];
    reconcile_body(r, I.g, blockIdx.x - I.block0, nblk, I.mask);
}

// one block per item
__global__ void __launch_bounds__(1024) k_fill_batch(const ReconcileArgs* tmpl, const BatchLaunch bl)
{
    const BatchItem I = bl.item[blockIdx.x];
    const ReconcileArgs r = tmpl[I.rep * kMaxSpecies + I.sel];
    fill_body(r, I.mask);
}

// one block per item
__global__ void __launch_bounds__(1024) k_births_batch(const EventArgs* tmpl, const BatchLaunch bl)
{
    const BatchItem I = bl.item[blockIdx.x];
    const EventArgs a = tmpl[I.rep * kMaxSpecies + I.sel];
    births_body(a);
}

void launch_claim_batch(const EventArgs* tmpl, const BatchLaunch& bl, int threads, cudaStream_t st)
{
    k_claim_batch<<<bl.total_blocks, threads, 0, st>>>(tmpl, bl);
}

void launch_commit_batch(const EventArgs* tmpl, const BatchLaunch& bl, int threads, cudaStream_t st)
{
    k_commit_batch<<<bl.total_blocks, threads, 0, st>>>(tmpl, bl);
}

void launch_reconcile_batch(const ReconcileArgs* tmpl, const BatchLaunch& bl, int threads, cudaStream_t st)
{
    k_reconcile_batch<<<bl.total_blocks, threads, 0, st>>>(tmpl, bl);
}

void launch_fill_batch(const ReconcileArgs* tmpl, const BatchLaunch& bl, cudaStream_t st)
{
    k_fill_batch<<<bl.n, 1024, 0, st>>>(tmpl, bl);
}

void launch_births_batch(const EventArgs* tmpl, const BatchLaunch& bl, cudaStream_t st)
{
    static bool configured = false;
    const int smem = kBirthSortMax * (int)sizeof(unsigned long long);
    if (!configured) {
        cudaFuncSetAttribute(k_births_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        configured = true;
    }
    k_births_batch<<<bl.n, 1024, smem, st>>>(tmpl, bl);
}

#include "psc_tiles.cuh"
#include "psc_slab.cuh"
#include "psc_subvol.cuh"

}  // namespace psc
