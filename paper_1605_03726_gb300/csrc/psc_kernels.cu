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
__constant__ uint32_t c_stencil[5];

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
    static uint32_t h[5];
    h[0] = pack_offsets(di0); h[1] = pack_offsets(di1);
    h[2] = pack_offsets(dj0); h[3] = pack_offsets(dj1);
    h[4] = pack_offsets(dk);
    cudaMemcpyToSymbolAsync(c_stencil, h, sizeof(h), 0, cudaMemcpyHostToDevice, st);
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

// Neighbour d of (i, j, k); false if it lies behind a reflective wall.
// wrap receives the change of the packed 16-bit wrap counters.
__device__ __forceinline__ bool neighbor(const Geometry& G, int32_t i, int32_t j, int32_t k, int d,
                                         int32_t& t, uint64_t& wrap)
{
    const uint32_t s0 = c_stencil[0], s1 = c_stencil[1], s2 = c_stencil[2], s3 = c_stencil[3],
                   s4 = c_stencil[4];
    const uint32_t wi = ((j + k) & 1) ? s1 : s0;
    const uint32_t wj = (k & 1) ? s3 : s2;
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
    t = ti + G.ni * (tj + G.nj * tk);
    wrap = w;
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
// vacancy mirror and claim tables
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool occupied(const uint32_t* bits, uint32_t v)
{
    return (bits[v >> 5] >> (v & 31u)) & 1u;
}

__device__ __forceinline__ void bit_set(uint32_t* bits, uint32_t v)
{
    atomicOr(&bits[v >> 5], 1u << (v & 31u));
}

__device__ __forceinline__ void bit_clear(uint32_t* bits, uint32_t v)
{
    atomicAnd(&bits[v >> 5], ~(1u << (v & 31u)));
}

__device__ __forceinline__ uint32_t slot_of(uint32_t t, uint32_t hash_bits)
{
    return (t * 2654435761u) >> (32u - hash_bits);     // Fibonacci hashing
}

// Claim voxel t for molecule id: the slot for t ends up holding the lowest id.
template <bool HASH>
__device__ __forceinline__ void claim(const EventArgs& a, uint32_t t, uint32_t id)
{
    if (!HASH) {
        atomicMin(&a.ct.direct[t], id);
        return;
    }
    const uint32_t mask = (1u << a.ct.hash_bits) - 1u;
    const uint64_t mine = ((uint64_t)t << 32) | id;
    uint32_t h = slot_of(t, a.ct.hash_bits);
    uint64_t cur = __ldcg((const unsigned long long*)&a.ct.hash[h]);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        if (cur == kEmptySlot) {
            const unsigned long long prev =
                atomicCAS((unsigned long long*)&a.ct.hash[h], (unsigned long long)kEmptySlot,
                          (unsigned long long)mine);
            if (prev == kEmptySlot) return;
            cur = prev;
        }
        if ((uint32_t)(cur >> 32) == t) {
            // same voxel: the slot's key never changes within the event, so the
            // 64-bit minimum is the minimum over ids
            if ((uint32_t)cur > id) atomicMin((unsigned long long*)&a.ct.hash[h], (unsigned long long)mine);
            return;
        }
        h = (h + 1u) & mask;
        cur = __ldcg((const unsigned long long*)&a.ct.hash[h]);
    }
    atomicOr(&a.sc->err, kErrClaimTableFull);
}

// Did molecule id win voxel t?  (Direct mode: the winner resets the word, which
// every loser then reads as "not mine".)
template <bool HASH>
__device__ __forceinline__ bool won(const EventArgs& a, uint32_t t, uint32_t id)
{
    if (!HASH) {
        if (a.ct.direct[t] != id) return false;
        a.ct.direct[t] = kNoClaim;
        return true;
    }
    const uint32_t mask = (1u << a.ct.hash_bits) - 1u;
    uint32_t h = slot_of(t, a.ct.hash_bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint64_t cur = __ldcg((const unsigned long long*)&a.ct.hash[h]);
        if (cur == kEmptySlot) return false;
        if ((uint32_t)(cur >> 32) == t) return (uint32_t)cur == id;
        h = (h + 1u) & mask;
    }
    return false;
}

// ---------------------------------------------------------------------------
// claim
// ---------------------------------------------------------------------------
template <bool GENERAL, bool HASH>
__global__ void __launch_bounds__(256) k_claim(const EventArgs a)
{
    const int32_t n = *a.count;
    if (blockIdx.x == 0 && threadIdx.x < kMaxSpecies) a.sc->tmp_count[threadIdx.x] = 0;
    unsigned long long n_att = 0, n_col = 0, n_acc = 0, n_fire = 0;
    const uint32_t c2 = ((uint32_t)a.s << 4) | kTagEvent;
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int idx = base + threadIdx.x;
        if (idx >= n) continue;
        const uint32_t v = (uint32_t)a.list.vox[idx];
        const uint32_t id = a.list.ids[idx];
        int32_t i, j, k;
        decode(a.geo, v, i, j, k);
        uint32_t u[4];
        philox(id, a.g, c2, 0u, a.key0, a.key1, u);
        ++n_att;
        if (GENERAL) {
            const ModelDev* M = a.model;
            if (M->n_fo[a.s] > 0 && (uint64_t)u[2] < M->T_fire[a.s]) {
                ++n_fire;
                const int r = pick_first_order(M, a.s, u[3]);
                if (M->rx[r].np == 2) {
                    // second product: uniform pick among neighbours vacant now
                    int c = 0;
                    for (int d = 0; d < 12; ++d) {
                        int32_t t; uint64_t w;
                        if (neighbor(a.geo, i, j, k, d, t, w) && !occupied(a.bits, t)) ++c;
                    }
                    if (c > 0) {
                        int want = (int)__umulhi(u[0], (uint32_t)c);
                        for (int d = 0; d < 12; ++d) {
                            int32_t t; uint64_t w;
                            if (neighbor(a.geo, i, j, k, d, t, w) && !occupied(a.bits, t)) {
                                if (want == 0) { claim<HASH>(a, (uint32_t)t, id); break; }
                                --want;
                            }
                        }
                    }
                }
                continue;
            }
        }
        const int d = (int)__umulhi(u[0], 12u);
        int32_t t; uint64_t w;
        if (!neighbor(a.geo, i, j, k, d, t, w)) continue;
        if (!occupied(a.bits, (uint32_t)t)) {
            claim<HASH>(a, (uint32_t)t, id);
        } else if (GENERAL) {
            const uint16_t o = a.occ[t];
            if (o != 0 && o != kBlocked) {
                const int r = a.model->pair[a.s][o - 1];
                if (r >= 0) {
                    ++n_col;
                    if ((uint64_t)u[1] < a.model->rx[r].T) {
                        ++n_acc;
                        claim<HASH>(a, (uint32_t)t, id);
                    }
                }
            }
        }
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

// ---------------------------------------------------------------------------
// commit
// ---------------------------------------------------------------------------
template <bool GENERAL, bool HASH>
__global__ void __launch_bounds__(256) k_commit(const EventArgs a)
{
    const int32_t n = *a.count;
    unsigned long long n_hop = 0, n_r2 = 0, n_r1 = 0;
    const uint32_t c2 = ((uint32_t)a.s << 4) | kTagEvent;
    const uint16_t self = (uint16_t)(a.s + 1);
    const int stride = gridDim.x * blockDim.x;
    if (HASH) {
        // empty the table of the previous event for the next one
        for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < a.ct.clear_n; x += stride)
            a.ct.clear[x] = kEmptySlot;
    }
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int idx = base + threadIdx.x;
        if (idx >= n) continue;
        const uint32_t v = (uint32_t)a.list.vox[idx];
        const uint32_t id = a.list.ids[idx];
        int32_t i, j, k;
        decode(a.geo, v, i, j, k);
        uint32_t u[4];
        philox(id, a.g, c2, 0u, a.key0, a.key1, u);
        if (GENERAL) {
            const ModelDev* M = a.model;
            if (M->n_fo[a.s] > 0 && (uint64_t)u[2] < M->T_fire[a.s]) {
                const ReactionDev R = M->rx[pick_first_order(M, a.s, u[3])];
                if (R.np == 2) {
                    // the neighbour this molecule claimed, if it won it
                    for (int d = 0; d < 12; ++d) {
                        int32_t t; uint64_t w;
                        if (!neighbor(a.geo, i, j, k, d, t, w) || occupied(a.bits, (uint32_t)t)) continue;
                        if (!won<HASH>(a, (uint32_t)t, id)) continue;
                        a.occ[v] = (uint16_t)(R.p0 + 1);
                        a.occ[t] = (uint16_t)(R.p1 + 1);
                        bit_set(a.bits, (uint32_t)t);
                        const int slot = atomicAdd(&a.sc->births, 1);
                        if (slot < a.births_cap) {
                            Birth b;
                            b.parent = id; b.t = t; b.species = R.p1; b.pad = 0;
                            b.img = img_add(a.list.img[idx], w);
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
                        bit_clear(a.bits, v);
                    }
                    ++n_r1;
                }
                continue;
            }
        }
        const int d = (int)__umulhi(u[0], 12u);
        int32_t t; uint64_t w;
        if (!neighbor(a.geo, i, j, k, d, t, w)) continue;
        if (!won<HASH>(a, (uint32_t)t, id)) continue;       // lost, or never claimed
        const uint16_t o = GENERAL ? a.occ[t] : (uint16_t)0;
        if (!GENERAL || !occupied(a.bits, (uint32_t)t)) {
            // move (Sec. 2.3)
            bit_clear(a.bits, v);
            bit_set(a.bits, (uint32_t)t);
            if (a.live) {
                a.occ[t] = self;
                a.occ[v] = 0;
            }
            a.list.vox[idx] = t;
            if (w) a.list.img[idx] = img_add(a.list.img[idx], w);
            ++n_hop;
        } else {
            // accepted collision with partner o - 1 (Sec. 2.4.2): first
            // product on the partner's voxel, second on the mover's
            const ReactionDev R = a.model->rx[a.model->pair[a.s][o - 1]];
            if (R.np >= 1) {
                a.occ[t] = (uint16_t)(R.p0 + 1);
            } else {
                a.occ[t] = 0;
                bit_clear(a.bits, (uint32_t)t);
            }
            if (R.np == 2) {
                a.occ[v] = (uint16_t)(R.p1 + 1);
            } else {
                a.occ[v] = 0;
                bit_clear(a.bits, v);
            }
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
// reconcile: bring the list of species x in line with the grid after an event
// with reactions.  An entry whose voxel holds x stays; one whose voxel holds
// species y (a product that inherited this molecule's identity) moves to y's
// list; one whose voxel is empty is dropped.  Species with reactions always
// keep their codes in occ, and a vacant voxel never keeps the code of one, so
// "occupied and code y + 1" identifies y exactly.
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

__global__ void __launch_bounds__(256) k_reconcile(const ReconcileArgs r)
{
    const int32_t n = r.sc->counts[r.x];
    const uint16_t self = (uint16_t)(r.x + 1);
    const int stride = gridDim.x * blockDim.x;
    for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
        const int idx = base + threadIdx.x;
        const bool valid = idx < n;
        int32_t v = 0; uint32_t id = 0; uint64_t img = 0; uint16_t o = 0;
        if (valid) {
            v = r.list.vox[idx];
            id = r.list.ids[idx];
            img = r.list.img[idx];
            o = ((r.bits[(uint32_t)v >> 5] >> ((uint32_t)v & 31u)) & 1u) ? r.occ[v] : (uint16_t)0;
        }
        const bool keep = valid && o == self;
        const int slot = warp_alloc(&r.sc->tmp_count[r.x], keep);
        if (keep) {
            r.tmp.vox[slot] = v;
            r.tmp.ids[slot] = id;
            r.tmp.img[slot] = img;
        } else if (valid && o != 0 && o != kBlocked) {
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

__global__ void __launch_bounds__(256) k_copyback(const ReconcileArgs r)
{
    const int32_t m = r.sc->tmp_count[r.x];
    if (blockIdx.x == 0 && threadIdx.x == 0) r.sc->counts[r.x] = m;
    const int stride = gridDim.x * blockDim.x;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < m; idx += stride) {
        r.list.vox[idx] = r.tmp.vox[idx];
        r.list.ids[idx] = r.tmp.ids[idx];
        r.list.img[idx] = r.tmp.img[idx];
    }
}

void launch_reconcile(const ReconcileArgs& r, int blocks, int threads, cudaStream_t st)
{
    k_reconcile<<<blocks, threads, 0, st>>>(r);
}

void launch_copyback(const ReconcileArgs& r, int blocks, int threads, cudaStream_t st)
{
    k_copyback<<<blocks, threads, 0, st>>>(r);
}

// ---------------------------------------------------------------------------
// births: one block sorts the births of this event by parent id (bitonic, in
// shared memory) and hands out ids next_id, next_id + 1, ... in that order.
// ---------------------------------------------------------------------------
constexpr int kBirthSortMax = 8192;

__global__ void __launch_bounds__(1024) k_births(const EventArgs a)
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
// the mirror says occupied, zero elsewhere; species without reactions are
// written afterwards from their lists (they do not keep codes while moving)
__global__ void k_materialize(uint16_t* out, const uint16_t* occ, const uint32_t* bits, int64_t V)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        out[v] = ((bits[v >> 5] >> (v & 31)) & 1u) ? occ[v] : (uint16_t)0;
}

void launch_materialize(uint16_t* out, const uint16_t* occ, const uint32_t* bits, int64_t V, int blocks,
                        cudaStream_t st)
{
    k_materialize<<<blocks, 256, 0, st>>>(out, occ, bits, V);
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

// placement key of every voxel: word 0 of Philox(seed; v, 0, 1, 0)
__global__ void k_populate_keys(uint32_t* keys, uint32_t* vals, uint32_t V, uint32_t key0, uint32_t key1)
{
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        uint32_t u[4];
        philox(v, 0u, kTagPopulate, 0u, key0, key1, u);
        keys[v] = u[0];
        vals[v] = v;
    }
}

void launch_populate_keys(uint32_t* keys, uint32_t* vals, uint32_t V, uint32_t key0, uint32_t key1,
                          int blocks, cudaStream_t st)
{
    k_populate_keys<<<blocks, 256, 0, st>>>(keys, vals, V, key0, key1);
}

struct Offsets {
    int64_t off[kMaxSpecies + 1];
};

// rank r of the sorted voxels goes to the species whose range holds r
__global__ void k_populate_scatter(const uint32_t* sorted_vox, int64_t n_total, Offsets o, int n_species,
                                   uint16_t* occ, uint32_t* bits, const ModelDev* model)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_total;
         r += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
        while (s + 1 < n_species && r >= o.off[s + 1]) ++s;
        const uint32_t v = sorted_vox[r];
        const int64_t a = r - o.off[s];
        occ[v] = (uint16_t)(s + 1);
        atomicOr(&bits[v >> 5], 1u << (v & 31u));
        const SpeciesList L = model->lists[s];
        L.vox[a] = (int32_t)v;
        L.ids[a] = (uint32_t)r;
        L.img[a] = 0ull;
    }
}

void launch_populate_scatter(const uint32_t* sorted_vox, int64_t n_total, const int64_t* offsets,
                             int n_species, uint16_t* occ, uint32_t* bits, const ModelDev* model,
                             int blocks, cudaStream_t st)
{
    Offsets o;
    for (int s = 0; s <= kMaxSpecies; ++s) o.off[s] = s <= n_species ? offsets[s] : offsets[n_species];
    k_populate_scatter<<<blocks, 256, 0, st>>>(sorted_vox, n_total, o, n_species, occ, bits, model);
}

// Morton (Z-order) key of the voxel of each list entry, 10 bits per axis
__device__ __forceinline__ uint32_t spread3(uint32_t x)
{
    x &= 0x3FFu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void k_morton_keys(const SpeciesList L, const int32_t* count, Geometry G, int shift,
                              uint32_t* keys, uint32_t* vals)
{
    const int32_t n = *count;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x) {
        int32_t i, j, k;
        decode(G, (uint32_t)L.vox[idx], i, j, k);
        keys[idx] = spread3((uint32_t)i >> shift) | (spread3((uint32_t)j >> shift) << 1) |
                    (spread3((uint32_t)k >> shift) << 2);
        vals[idx] = (uint32_t)idx;
    }
}

void launch_morton_keys(const SpeciesList& list, const int32_t* count, const Geometry& geo,
                        uint32_t* keys, uint32_t* vals, int blocks, cudaStream_t st)
{
    int maxdim = geo.ni > geo.nj ? geo.ni : geo.nj;
    if (geo.nk > maxdim) maxdim = geo.nk;
    int shift = 0;
    while ((maxdim - 1) >> shift >= 1024) ++shift;
    k_morton_keys<<<blocks, 256, 0, st>>>(list, count, geo, shift, keys, vals);
}

__global__ void k_permute(const SpeciesList src, const SpeciesList dst, const uint32_t* perm, const int32_t* count)
{
    const int32_t n = *count;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const uint32_t p = perm[r];
        dst.vox[r] = src.vox[p];
        dst.ids[r] = src.ids[p];
        dst.img[r] = src.img[p];
    }
}

void launch_permute(const SpeciesList& src, const SpeciesList& dst, const uint32_t* perm,
                    const int32_t* count, int blocks, cudaStream_t st)
{
    k_permute<<<blocks, 256, 0, st>>>(src, dst, perm, count);
}

__global__ void k_copy_list(const SpeciesList src, const SpeciesList dst, const int32_t* count)
{
    const int32_t n = *count;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        dst.vox[r] = src.vox[r];
        dst.ids[r] = src.ids[r];
        dst.img[r] = src.img[r];
    }
}

void launch_copy_list(const SpeciesList& src, const SpeciesList& dst, const int32_t* count,
                      int blocks, cudaStream_t st)
{
    k_copy_list<<<blocks, 256, 0, st>>>(src, dst, count);
}

}  // namespace psc
