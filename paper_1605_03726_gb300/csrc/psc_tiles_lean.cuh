// psc_tiles_lean.cuh -- the tile kernel for its common case: HCP lattices of
// whole mirror bricks (ni, nj multiples of 4, nk even) cut into boxes at
// least two bricks thick, never a single box along a periodic axis.  Part of
// psc_kernels.cu's translation unit (after psc_tiles.cuh, whose plan, bucket,
// inbox, neighbour-wait and hand-over helpers it shares).
//
// Same owner-computes protocol and the same results as k_tile_run (Sec. 2.3,
// synchronous rule), with less work per molecule:
//   - every (place c of the molecule in its brick word, direction d) is looked
//     up in tables built once per launch in shared memory: the packed step of
//     the box coordinates, and the eight-word window around the target with
//     the masks of the target and of its twelve neighbours (Sec. 2.1) minus
//     the mover itself, so "the target is vacant and nobody else can reach
//     it" is one OR over eight masked box words;
//   - words behind a reflective wall hold all ones in the box, so no hop
//     needs a bounds test (a wall voxel looks occupied: the hop fails, and a
//     target next to a wall takes the claim path, which gives the same result);
//   - the halo refresh reads a per-box table of (box word, global word) pairs
//     built once per launch from per-axis tables of global brick coordinates,
//     instead of per-word wrap arithmetic at every event;
//   - a contested target whose twelve neighbours all lie in the region can
//     only be wanted by molecules of this box: its claim goes to a table in
//     shared memory (lowest id wins, as in the global words) and is read back
//     inline in the commit phase; targets nearer the region's faces are
//     claimed in the global words as before;
//   - the commit phase handles every molecule in one pass: hops inside the
//     box update the box (and, for the outermost brick layer, the global
//     mirror), global claim words are read back in batches of loads, and
//     departures go to the outbox (one inbox atomic per destination box and
//     warp when it is flushed), with no deferred queue;
//   - whether a word is in the region's outermost brick layer comes from a
//     bitmap in shared memory; the next chunk's bucket entries load while one
//     is processed.

constexpr uint32_t kLeanOff = 4u | (4u << 11) | (2u << 22);   // region -> box coordinates

struct LeanShared {
    uint32_t* box;
    unsigned long long* ctab;  // block-local claims: (packed target << 32 | lowest id), all ones = empty
    uint4* tmask;              // [kLeanEntries][2]: masks of the eight-word window
    int32_t* tstep;            // [kLeanEntries]: packed step dx + 2048 dy + 4194304 dz
    int32_t* tbase;            // [kLeanEntries]: first window word minus the mover's word
    int32_t* o_t;              // outbox: departures of an event
    uint32_t* o_id;
    int32_t* o_q;
    int32_t* hx;               // global brick coordinate of box word coordinate x (-1: wall)
    int32_t* hy;
    int32_t* hz;
    uint32_t* obits;           // bit w: box word w is in the region's outermost brick layer
    uint8_t* own;              // owner tables
};

__device__ __forceinline__ LeanShared lean_shared(uint32_t* smem, const TilePlan& P, const TileBox& b)
{
    LeanShared S;
    S.box = smem;
    S.ctab = reinterpret_cast<unsigned long long*>(smem + ((P.box_words + 3) & ~3));
    S.tmask = reinterpret_cast<uint4*>(S.ctab + (1 << kLeanClaimBits));
    S.tstep = reinterpret_cast<int32_t*>(S.tmask + 2 * kLeanEntries);
    S.tbase = S.tstep + kLeanEntries;
    S.o_t = S.tbase + kLeanEntries;
    S.o_id = reinterpret_cast<uint32_t*>(S.o_t + kLeanOutbox);
    S.o_q = S.o_t + 2 * kLeanOutbox;
    S.hx = S.o_t + 3 * kLeanOutbox;
    S.hy = S.hx + b.BI;
    S.hz = S.hy + b.BJ;
    const int halo_tables = ((P.ei + 2) + (P.ej + 2) + (P.ek + 2) + 3) & ~3;
    S.obits = reinterpret_cast<uint32_t*>(S.hx + halo_tables);
    S.own = reinterpret_cast<uint8_t*>(S.obits + ((P.box_words + 31) >> 5));
    return S;
}

// box word index and place of packed box coordinates bx | by << 11 | bz << 22
__device__ __forceinline__ int lean_word(uint32_t p, int BI, int BIJ)
{
    return (int)(p >> 23) * BIJ + (int)((p >> 13) & 0x1FFu) * BI + (int)((p >> 2) & 0x1FFu);
}
__device__ __forceinline__ uint32_t lean_place(uint32_t p)
{
    return (p & 3u) | ((p >> 9) & 0xCu) | ((p >> 18) & 0x10u);
}

// global mirror word of the region word holding packed coordinates p
__device__ __forceinline__ int64_t lean_gword(uint32_t p, const TilePlan& P, int64_t gbase)
{
    const int wx = (int)((p >> 2) & 0x1FFu), wy = (int)((p >> 13) & 0x1FFu), wz = (int)(p >> 23);
    return gbase + ((int64_t)wz * P.nbj + wy) * P.nbi + wx;
}

__device__ void lean_build_tables(const TileBox& b, const TilePlan& P, const Geometry& G, const LeanShared& S)
{
    const int BI = b.BI, BIJ = b.BI * b.BJ;
    for (int e = threadIdx.x; e < kLeanEntries; e += blockDim.x) {
        const int c = e / 12, d = e - 12 * c;
        const int x = 4 + (c & 3), y = 4 + ((c >> 2) & 3), z = 2 + ((c >> 4) & 1);
        int dx, dy, dz;
        tile_step(d, y, z, -1, dx, dy, dz);
        const int tx = x + dx, ty = y + dy, tz = z + dz;
        S.tstep[e] = dx + dy * 2048 + dz * 4194304;
        const int wx0 = (tx - 1) >> 2, wy0 = (ty - 1) >> 2, wz0 = (tz - 1) >> 1;
        S.tbase[e] = (wz0 - (z >> 1)) * BIJ + (wy0 - (y >> 2)) * BI + (wx0 - (x >> 2));
        uint32_t m[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
        for (int d2 = -1; d2 < 12; ++d2) {
            int ex = 0, ey = 0, ez = 0;
            if (d2 >= 0) tile_step(d2, ty, tz, -1, ex, ey, ez);
            const int nx = tx + ex, ny = ty + ey, nz = tz + ez;
            if (nx == x && ny == y && nz == z) continue;          // the mover itself
            const int q = ((nx >> 2) - wx0) | (((ny >> 2) - wy0) << 1) | (((nz >> 1) - wz0) << 2);
            m[q] |= 1u << ((nx & 3) | ((ny & 3) << 2) | ((nz & 1) << 4));
        }
        S.tmask[2 * e] = make_uint4(m[0], m[1], m[2], m[3]);
        S.tmask[2 * e + 1] = make_uint4(m[4], m[5], m[6], m[7]);
    }
    // per-axis global brick coordinates of the box word coordinates, wrapped
    // along periodic axes, -1 behind a reflective wall
    for (int q = threadIdx.x; q < b.BI + b.BJ + b.BK; q += blockDim.x) {
        int a, w, first, nb;
        if (q < b.BI) { a = 0; w = q; first = b.bi0; nb = P.nbi; }
        else if (q < b.BI + b.BJ) { a = 1; w = q - b.BI; first = b.bj0; nb = P.nbj; }
        else { a = 2; w = q - b.BI - b.BJ; first = b.bk0; nb = P.nbk; }
        int g = first - 1 + w;
        if (g < 0 || g >= nb) g = (G.bflags & (1u << a)) ? (g < 0 ? g + nb : g - nb) : -1;
        S.hx[q] = g;                       // hx, hy, hz are consecutive
    }
}

// The halo (box words outside the region) is refreshed from the global
// mirror at every event; words behind a reflective wall are all ones and never
// change.  Halo word q: first the two z faces (full planes), then the full rows
// of the two y faces, then the end words of the other rows.  Each block writes
// the (box word, global word) pair of every halo word into its part of a table
// once per launch; an event then reads its pairs instead of recomputing them.
// A thread takes the words q0 + h * blockDim.x, h < kLeanHalo, of a chunk, whose
// loads go out together.
constexpr int kLeanHalo = 8;
constexpr uint32_t kLeanWall = ~0u;         // global word of a halo word behind a wall

__device__ __forceinline__ int lean_halo_total(const TileBox& b)
{
    return 2 * b.BI * b.BJ + 2 * (b.BK - 2) * b.BI + 2 * (b.BK - 2) * (b.BJ - 2);
}

// (box word, global word or kLeanWall) of halo word q
__device__ __forceinline__ uint2 lean_halo_pair(const TilePlan& P, const TileBox& b, const LeanShared& S,
                                                const FastDiv& div_bi, const FastDiv& div_bj2, int q)
{
    const int BI = b.BI, BJ = b.BJ, BK = b.BK, BIJ = BI * BJ;
    const int n_z = 2 * BIJ;
    const int n_y = n_z + 2 * (BK - 2) * BI;
    int wx, wy, wz;
    if (q < n_z) {
        const int f = q >= BIJ ? 1 : 0;
        const int r = q - f * BIJ;
        wy = (int)fdiv((uint32_t)r, div_bi);
        wx = r - wy * BI;
        wz = f ? BK - 1 : 0;
    } else if (q < n_y) {
        const int r2 = q - n_z;
        const int row = (int)fdiv((uint32_t)r2, div_bi);
        wx = r2 - row * BI;
        wz = 1 + (row >> 1);
        wy = (row & 1) ? BJ - 1 : 0;
    } else {
        const int r3 = q - n_y;
        const int col = (int)fdiv((uint32_t)r3, div_bj2);
        wy = 1 + r3 - col * (BJ - 2);
        wz = 1 + (col >> 1);
        wx = (col & 1) ? BI - 1 : 0;
    }
    const int gi = S.hx[wx], gj = S.hy[wy], gk = S.hz[wz];
    const uint32_t g = (gi | gj | gk) >= 0 ? (uint32_t)(((int64_t)gk * P.nbj + gj) * P.nbi + gi) : kLeanWall;
    return make_uint2((uint32_t)((wz * BJ + wy) * BI + wx), g);
}

// Launch prologue: the block's table, and every halo word (walls included)
__device__ __forceinline__ void lean_halo_init(const TileArgs& A, int r, const TileBox& b, const LeanShared& S,
                                               const FastDiv& div_bi, const FastDiv& div_bj2)
{
    const int total = lean_halo_total(b);
    uint2* tab = A.halo_tab + (int64_t)r * A.halo_cap;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const uint2 e = lean_halo_pair(A.plan, b, S, div_bi, div_bj2, q);
        tab[q] = e;                       // read back only by this thread (same q stride)
        S.box[e.x] = e.y == kLeanWall ? ~0u : __ldcg(&A.ev.bits[e.y]);
    }
}

// the table entries of chunk q0 (kLeanWall pairs past the end)
__device__ __forceinline__ void lean_halo_fetch(const TileArgs& A, int r, int total, int q0, uint2 (&e)[kLeanHalo])
{
    const uint2* tab = A.halo_tab + (int64_t)r * A.halo_cap;
#pragma unroll
    for (int h = 0; h < kLeanHalo; ++h) {
        const int q = q0 + h * blockDim.x;
        e[h] = q < total ? __ldcg(reinterpret_cast<const uint2*>(tab) + q) : make_uint2(0u, kLeanWall);
    }
}

__device__ __forceinline__ void lean_halo_load(const uint32_t* bits, const uint2 (&e)[kLeanHalo],
                                               uint32_t (&val)[kLeanHalo])
{
#pragma unroll
    for (int h = 0; h < kLeanHalo; ++h) val[h] = e[h].y != kLeanWall ? __ldcg(&bits[e[h].y]) : 0u;
}

__device__ __forceinline__ void lean_halo_store(const LeanShared& S, const uint2 (&e)[kLeanHalo],
                                                const uint32_t (&val)[kLeanHalo])
{
#pragma unroll
    for (int h = 0; h < kLeanHalo; ++h)
        if (e[h].y != kLeanWall) S.box[e[h].x] = val[h];
}

// A molecule of the box (packed box coordinates p, place c) moves to packed
// box coordinates t inside its region: box bits, and the global mirror for
// words of the outermost layer.
__device__ __forceinline__ void lean_move_inside(const TileArgs& A, const LeanShared& S, uint32_t* box, int BI,
                                                 int BIJ, int64_t gbase, uint32_t p, uint32_t c, uint32_t t)
{
    const int wv = lean_word(p, BI, BIJ), wt = lean_word(t, BI, BIJ);
    const uint32_t mv = 1u << c, mt = 1u << lean_place(t);
    const bool vo = (S.obits[wv >> 5] >> (wv & 31)) & 1u, to = (S.obits[wt >> 5] >> (wt & 31)) & 1u;
    if (wv == wt) {
        atomicXor(&box[wv], mv | mt);
        if (vo) atomicXor(&A.ev.bits[lean_gword(p, A.plan, gbase)], mv | mt);
    } else {
        atomicXor(&box[wv], mv);
        atomicXor(&box[wt], mt);
        if (vo) atomicXor(&A.ev.bits[lean_gword(p, A.plan, gbase)], mv);
        if (to) atomicXor(&A.ev.bits[lean_gword(t, A.plan, gbase)], mt);
    }
}

// A molecule (packed box coordinates p, place c) leaves its region for
// packed box coordinates t: its bit leaves the box and the global mirror, the
// target's bit is set in the global mirror (the owner's box picks it up with
// the arrival), wrap counters follow a periodic wrap, and the molecule goes
// to the outbox (or straight to the inbox when the outbox is full).
__device__ __forceinline__ void lean_depart(const TileArgs& A, const TileBox& b, const LeanShared& S, int BI,
                                            int BIJ, int64_t gbase, int* s_out_n, uint32_t p, uint32_t c, uint32_t t,
                                            uint32_t id)
{
    const Geometry& G = A.ev.geo;
    int32_t gi, gj, gk;
    uint64_t wr;
    tile_global(G, b, (int)(t & 0x7FFu), (int)((t >> 11) & 0x7FFu), (int)(t >> 22), gi, gj, gk, wr);
    if (wr) {
        uint64_t* wp = &A.img_id[id - A.id_lo];
        *wp = img_add(*wp, wr);
    }
    const uint32_t mv = 1u << c;
    atomicXor(&S.box[lean_word(p, BI, BIJ)], mv);
    atomicXor(&A.ev.bits[lean_gword(p, A.plan, gbase)], mv);   // the source is in the outermost layer
    const BitPos gt = bitpos(G, gi, gj, gk);
    atomicXor(&A.ev.bits[gt.word], gt.mask);
    const int q = tile_region_of(A.plan, S.own, gi, gj, gk);
    const int32_t tv = gi + G.ni * (gj + G.nj * gk);
    const int o = atomicAdd(s_out_n, 1);
    if (o < kLeanOutbox) {
        S.o_t[o] = tv;
        S.o_id[o] = id;
        S.o_q[o] = q;
    } else {
        const int cap = A.plan.cap;
        const int slot = atomicAdd(&A.in_cnt[q], 1);
        if (slot < cap) {
            A.in_vox[(int64_t)q * cap + slot] = tv;
            A.in_ids[(int64_t)q * cap + slot] = id;
        } else {
            atomicOr(&A.ev.sc->err, kErrListOverflow);
        }
    }
}

// Claim target t (packed box coordinates) for molecule id in the block-local
// table: linear probing from a hash of t over at most 8 slots.  Returns the
// slot, or -1 when all 8 hold other targets (the claim then goes to the
// global words).  Slots only go from empty to a target within an event, so
// every claimant of t takes the same branch.
constexpr int kLeanProbes = 8;
__device__ __forceinline__ int lean_claim_local(unsigned long long* tab, uint32_t t, uint32_t id)
{
    const unsigned long long v = ((unsigned long long)t << 32) | id;
    uint32_t slot = (t * 0x9E3779B1u) >> (32 - kLeanClaimBits);
    for (int probe = 0; probe < kLeanProbes; ++probe) {
        const unsigned long long old = atomicCAS(&tab[slot], kEmptySlot, v);
        if (old == kEmptySlot) return (int)slot;
        if ((uint32_t)(old >> 32) == t) {
            atomicMin(&tab[slot], v);
            return (int)slot;
        }
        slot = (slot + 1u) & ((1u << kLeanClaimBits) - 1u);
    }
    return -1;
}
constexpr uint32_t kLeanLocal = 0x20000000u;   // claimed in the local table (slot in bits 4-13)

// global voxel index of packed box coordinates t (a target next to the region)
__device__ __forceinline__ int32_t lean_voxel(const Geometry& G, const TileBox& b, uint32_t t)
{
    int32_t i, j, k;
    uint64_t wr;
    tile_global(G, b, (int)(t & 0x7FFu), (int)((t >> 11) & 0x7FFu), (int)(t >> 22), i, j, k, wr);
    return i + G.ni * (j + G.nj * k);
}

// End of a phase: once the whole block is done, publish flags[r] = value and
// wait until every neighbouring box (up to 26, across periodic wraps) has
// published at least value.  Two block barriers in all.  Bounded like the
// grid barrier; false (error raised) on time-out.  *s_ok is 1 from the launch
// on and becomes 0 only on a time-out, after which the kernel returns.
__device__ __forceinline__ bool lean_phase_sync(const TileArgs& A, uint32_t* flags, int r, uint32_t value,
                                                int* s_ok)
{
    const TilePlan& P = A.plan;
    const uint32_t bf = A.ev.geo.bflags;
    const uint32_t target = value + (A.barrier_phantom ? 0x40000000u : 0u);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(&flags[r], value);
    }
    if (threadIdx.x < 27 && threadIdx.x != 13) {
        int ri = r % P.pi + (int)(threadIdx.x % 3) - 1;
        int rj = (r / P.pi) % P.pj + (int)((threadIdx.x / 3) % 3) - 1;
        int rk = r / (P.pi * P.pj) + (int)(threadIdx.x / 9) - 1;
        bool skip = false;
        if (ri < 0 || ri >= P.pi) { if (bf & 1u) ri = (ri + P.pi) % P.pi; else skip = true; }
        if (rj < 0 || rj >= P.pj) { if (bf & 2u) rj = (rj + P.pj) % P.pj; else skip = true; }
        if (rk < 0 || rk >= P.pk) { if (bf & 4u) rk = (rk + P.pk) % P.pk; else skip = true; }
        if (!skip) {
            const volatile uint32_t* f = flags + (rk * P.pj + rj) * P.pi + ri;
            uint64_t t0 = 0;
            for (unsigned int spins = 0; *f < target; ++spins) {
                if ((spins & 1023u) == 0u) {
                    const uint64_t now = globaltimer_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > A.barrier_timeout_ns || spins >= kBarrierMaxSpins) {
                        atomicOr(&A.ev.sc->err, kErrBarrierTimeout);
                        *s_ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *s_ok != 0;
}

// Start of an event (after the neighbours' commits): the arrivals of the last
// event join the box and the bucket buffer `buf`, and (refresh) the halo is
// read again from the global mirror, in one pass with one block barrier.  The
// inbox count is reset afterwards by thread 0; senders write the inbox again
// only after this box publishes its next claim phase.
__device__ __forceinline__ void lean_ingest(const TileArgs& A, int r, const TileBox& b, const LeanShared& S, int& n,
                                            int buf, bool refresh, const uint2 (&first)[kLeanHalo])
{
    const int cap = A.plan.cap;
    const int m = min(*((volatile int32_t*)&A.in_cnt[r]), cap);
    const int64_t base = (int64_t)r * cap;
    // the first chunk of halo loads goes out before the arrivals are read
    const int total = refresh ? lean_halo_total(b) : 0;
    uint32_t val[kLeanHalo];
    if (refresh) lean_halo_load(A.ev.bits, first, val);
    for (int x = threadIdx.x; x < m; x += blockDim.x) {
        const int32_t t = __ldcg(&A.in_vox[base + x]);
        const uint32_t id = __ldcg(&A.in_ids[base + x]);
        int32_t i, j, k;
        decode(A.ev.geo, (uint32_t)t, i, j, k);
        int w;
        uint32_t mk;
        tile_local(b, i, j, k, w, mk);
        atomicOr(&S.box[w], mk);
        if (n + x < cap) {
            A.b_vox[buf][base + n + x] = (int32_t)tile_pack(i - 4 * b.bi0, j - 4 * b.bj0, k - 2 * b.bk0);
            A.b_ids[buf][base + n + x] = id;
        } else {
            atomicOr(&A.ev.sc->err, kErrListOverflow);
        }
    }
    if (refresh) {
        lean_halo_store(S, first, val);
        for (int q0 = threadIdx.x + kLeanHalo * blockDim.x; q0 < total; q0 += kLeanHalo * blockDim.x) {
            uint2 e[kLeanHalo];
            lean_halo_fetch(A, r, total, q0, e);
            lean_halo_load(A.ev.bits, e, val);
            lean_halo_store(S, e, val);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) A.in_cnt[r] = 0;
    n = min(n + m, cap);
}

// Claim-phase decision: bits 0-3 the direction, kTileMove (no claim needed)
// or kTileClaimed (claimed in the global words); neither: the hop fails.
__global__ void __launch_bounds__(kTileThreads, kTileBlocksPerSM) k_tile_lean(const TileArgs A)
{
    extern __shared__ uint32_t smem[];
    // s_misc: -, survivors, outbox entries, wait flag (1 until a wait times out), -, -
    __shared__ int s_misc[6];
    const EventArgs& a = A.ev;
    const Geometry& G = a.geo;
    const TilePlan& P = A.plan;
    const int r = blockIdx.x;
    const TileBox b = tile_box(P, r);
    const LeanShared S = lean_shared(smem, P, b);
    uint32_t* box = S.box;
    const int BI = b.BI, BIJ = b.BI * b.BJ;
    const int cap = P.cap;
    const int64_t base = (int64_t)r * cap;
    const uint32_t c2 = ((uint32_t)a.s << 4) | kTagEvent;
    uint32_t* claim = A.claim;
    const int64_t gbase = ((int64_t)(b.bk0 - 1) * P.nbj + (b.bj0 - 1)) * P.nbi + (b.bi0 - 1);
    const uint32_t rxn = 4u * (uint32_t)b.ei, ryn = 4u * (uint32_t)b.ej, rzn = 2u * (uint32_t)b.ek;
    const FastDiv div_bi = tile_fastdiv((uint32_t)b.BI), div_bj2 = tile_fastdiv((uint32_t)(b.BJ - 2));
    constexpr int U = 2;                                 // molecules whose memory operations go out together
    tile_build_owners(P, S.own);
    lean_build_tables(b, P, G, S);
    for (int q = threadIdx.x; q < (1 << kLeanClaimBits); q += blockDim.x) S.ctab[q] = kEmptySlot;
    for (int q = threadIdx.x; q < (P.box_words + 31) >> 5; q += blockDim.x) {
        uint32_t m = 0u;
        for (int z = 0; z < 32; ++z) {
            const int w = q * 32 + z;
            if (w >= b.BI * b.BJ * b.BK) break;
            const int wx = w % b.BI, wy = (w / b.BI) % b.BJ, wz = w / (b.BI * b.BJ);
            const bool inside = wx >= 1 && wx <= b.ei && wy >= 1 && wy <= b.ej && wz >= 1 && wz <= b.ek;
            const bool outer = wx == 1 || wx == b.ei || wy == 1 || wy == b.ej || wz == 1 || wz == b.ek;
            if (inside && outer) m |= 1u << z;
        }
        S.obits[q] = m;
    }
    if (threadIdx.x == 0) s_misc[3] = 1;
    __syncthreads();
    // region words from the global mirror, then the halo
    for (int q = threadIdx.x; q < b.ei * b.ej * b.ek; q += blockDim.x) {
        const int wx = 1 + q % b.ei, wy = 1 + (q / b.ei) % b.ej, wz = 1 + q / (b.ei * b.ej);
        box[(wz * b.BJ + wy) * BI + wx] = __ldcg(&a.bits[tile_region_word(P, b, wx, wy, wz)]);
    }
    lean_halo_init(A, r, b, S, div_bi, div_bj2);
    const int halo_total = lean_halo_total(b);
    int n = *((volatile int32_t*)&A.b_cnt[r]);
    // the scatter left voxel indices: store coordinates relative to the region
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        int32_t i, j, k;
        decode(G, (uint32_t)A.b_vox[0][base + x], i, j, k);
        A.b_vox[0][base + x] = (int32_t)tile_pack(i - 4 * b.bi0, j - 4 * b.bj0, k - 2 * b.bk0);
    }
    unsigned long long n_att = 0, n_hop = 0;
    uint2 halo_first[kLeanHalo];
    __syncthreads();
    for (int e = 0; e < A.n_events; ++e) {
        const uint32_t g = a.g + (uint32_t)e;
        const int cur = e & 1;
        const int32_t* bv = A.b_vox[cur] + base;
        const uint32_t* bi = A.b_ids[cur] + base;
        uint32_t* bs = A.b_state + base;
        if (e > 0) lean_ingest(A, r, b, S, n, cur, true, halo_first);   // after the neighbours' commits
        // ---- claim phase (the next chunk's bucket entries load while one is processed) ----
        uint32_t pv[U], pi_[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int x = u * blockDim.x + threadIdx.x;
            pv[u] = x < n ? (uint32_t)__ldcg(bv + x) : 0u;
            pi_[u] = x < n ? __ldcg(bi + x) : 0u;
        }
        for (int c0 = 0; c0 < n; c0 += U * blockDim.x) {
            uint32_t vv[U], ii[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                vv[u] = pv[u];
                ii[u] = pi_[u];
                const int x = c0 + (U + u) * blockDim.x + threadIdx.x;
                pv[u] = x < n ? (uint32_t)__ldcg(bv + x) : 0u;
                pi_[u] = x < n ? __ldcg(bi + x) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int xm = c0 + u * blockDim.x + threadIdx.x;
                if (xm >= n) continue;
                const uint32_t p = vv[u] + kLeanOff;
                uint32_t rnd[4];
                philox(ii[u], g, c2, 0u, a.key0, a.key1, rnd);
                const uint32_t d = __umulhi(rnd[0], 12u);
                const int e12 = (int)(lean_place(p) * 12u + d);
                const int w0 = lean_word(p, BI, BIJ) + S.tbase[e12];
                const uint4 m0 = S.tmask[2 * e12], m1 = S.tmask[2 * e12 + 1];
                const uint32_t busy = (box[w0] & m0.x) | (box[w0 + 1] & m0.y) | (box[w0 + BI] & m0.z) |
                                      (box[w0 + BI + 1] & m0.w) | (box[w0 + BIJ] & m1.x) |
                                      (box[w0 + BIJ + 1] & m1.y) | (box[w0 + BIJ + BI] & m1.z) |
                                      (box[w0 + BIJ + BI + 1] & m1.w);
                uint32_t st = d;
                if (busy == 0u) {
                    st |= kTileMove;                     // vacant, and only the mover is next to it
                } else {
                    const uint32_t t = p + (uint32_t)S.tstep[e12];
                    if (!(box[lean_word(t, BI, BIJ)] & (1u << lean_place(t)))) {
                        // vacant, but other molecules can reach it: the lowest id wins
                        int slot = -1;
                        if (((t & 0x7FFu) - 5u) < rxn - 2u && (((t >> 11) & 0x7FFu) - 5u) < ryn - 2u &&
                            ((t >> 22) - 3u) < rzn - 2u)
                            slot = lean_claim_local(S.ctab, t, ii[u]);   // all its neighbours are ours
                        if (slot >= 0) {
                            st |= kLeanLocal | ((uint32_t)slot << 4);
                        } else {
                            atomicMin(&claim[lean_voxel(G, b, t)], ii[u]);
                            st |= kTileClaimed;
                        }
                    }
                }
                bs[xm] = st;
            }
        }
        n_att += (unsigned long long)n;
        if (threadIdx.x == 0) {
            s_misc[1] = 0;
            s_misc[2] = 0;
        }
        // a claim word is touched only by boxes that are all neighbours of each other
        if (!lean_phase_sync(A, A.claimed, r, (uint32_t)(e + 1), &s_misc[3])) return;
        // ---- commit phase: every molecule in one pass ----
        int32_t* ov = A.b_vox[cur ^ 1] + base;
        uint32_t* oi = A.b_ids[cur ^ 1] + base;
        uint32_t qv[U], qi[U], qs[U];             // the next chunk, loading ahead
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int x = u * blockDim.x + threadIdx.x;
            qv[u] = x < n ? (uint32_t)__ldcg(bv + x) : 0u;
            qi[u] = x < n ? __ldcg(bi + x) : 0u;
            qs[u] = x < n ? __ldcg(bs + x) : 0u;
        }
        for (int c0 = 0; c0 < n; c0 += U * blockDim.x) {
            uint32_t vv[U], ii[U], ss[U], tt[U], rb[U];
            int32_t tv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                vv[u] = qv[u];
                ii[u] = qi[u];
                ss[u] = qs[u];
                const int x = c0 + (U + u) * blockDim.x + threadIdx.x;
                qv[u] = x < n ? (uint32_t)__ldcg(bv + x) : 0u;
                qi[u] = x < n ? __ldcg(bi + x) : 0u;
                qs[u] = x < n ? __ldcg(bs + x) : 0u;
            }
            // targets; the global claim words of contested targets near the faces go out together
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t p = vv[u] + kLeanOff;
                tt[u] = p + (uint32_t)S.tstep[lean_place(p) * 12u + (ss[u] & 15u)];
                tv[u] = -1;
                rb[u] = 0u;
                if (ss[u] & kTileClaimed) {
                    tv[u] = lean_voxel(G, b, tt[u]);
                    rb[u] = __ldcg(&claim[tv[u]]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int xm = c0 + u * blockDim.x + threadIdx.x;
                const uint32_t st = ss[u];
                uint32_t w = vv[u];
                bool keep = xm < n;
                bool win = (st & kTileMove) != 0u;
                if (st & kLeanLocal) {
                    win = (uint32_t)S.ctab[(st >> 4) & ((1u << kLeanClaimBits) - 1u)] == ii[u];
                } else if ((st & kTileClaimed) && rb[u] == ii[u]) {
                    win = true;
                    claim[tv[u]] = kNoClaim;             // the winner resets the word
                }
                if (keep && win) {
                    const uint32_t p = w + kLeanOff, t = tt[u];
                    const uint32_t c = lean_place(p);
                    ++n_hop;
                    if (((t & 0x7FFu) - 4u) < rxn && (((t >> 11) & 0x7FFu) - 4u) < ryn && ((t >> 22) - 2u) < rzn) {
                        lean_move_inside(A, S, box, BI, BIJ, gbase, p, c, t);
                        w = t - kLeanOff;
                    } else {
                        lean_depart(A, b, S, BI, BIJ, gbase, &s_misc[2], p, c, t, ii[u]);
                        keep = false;
                    }
                }
                tile_keep(keep, w, ii[u], &s_misc[1], ov, oi);
            }
        }
        __syncthreads();
        n = s_misc[1];
        // every read-back of the local table is done: empty it for the next event
        for (int q = threadIdx.x; q < (1 << kLeanClaimBits); q += blockDim.x) S.ctab[q] = kEmptySlot;
        // the outbox to the inboxes of the boxes the molecules entered
        {
            // one inbox atomic per destination box and warp
            const int m = min(s_misc[2], kLeanOutbox);
            for (int o0 = threadIdx.x & ~31; o0 < m; o0 += blockDim.x) {
                const int o = o0 + (threadIdx.x & 31);
                const bool has = o < m;
                const int q = has ? S.o_q[o] : -1;
                const unsigned peers = __match_any_sync(0xFFFFFFFFu, q);
                const int leader = __ffs(peers) - 1;
                const int lane = threadIdx.x & 31;
                int base0 = 0;
                if (has && lane == leader) base0 = atomicAdd(&A.in_cnt[q], __popc(peers));
                base0 = __shfl_sync(0xFFFFFFFFu, base0, leader);
                if (has) {
                    const int slot = base0 + __popc(peers & ((1u << lane) - 1u));
                    if (slot < cap) {
                        A.in_vox[(int64_t)q * cap + slot] = S.o_t[o];
                        A.in_ids[(int64_t)q * cap + slot] = S.o_id[o];
                    } else {
                        atomicOr(&a.sc->err, kErrListOverflow);
                    }
                }
            }
        }
        // the first chunk of the next halo refresh: its table entries load during the wait
        lean_halo_fetch(A, r, halo_total, threadIdx.x, halo_first);
        // halo bits, arrivals and reset claim words of every neighbour are out
        if (!lean_phase_sync(A, A.done, r, (uint32_t)(e + 1), &s_misc[3])) return;
    }
    // the last event's arrivals, then the region's bits back to the mirror
    if (A.n_events > 0) lean_ingest(A, r, b, S, n, A.n_events & 1, false, halo_first);
    for (int q = threadIdx.x; q < b.ei * b.ej * b.ek; q += blockDim.x) {
        const int wx = 1 + q % b.ei, wy = 1 + (q / b.ei) % b.ej, wz = 1 + q / (b.ei * b.ej);
        a.bits[tile_region_word(P, b, wx, wy, wz)] = box[(wz * b.BJ + wy) * BI + wx];
    }
    if (threadIdx.x == 0) A.b_cnt[r] = n;
    if (a.collect_stats) {
        if (threadIdx.x == 0) atomicAdd(&a.sc->stats[kStatAttempts], n_att);
        flush_stat(&a.sc->stats[kStatHops], n_hop);
    }
}

static cudaError_t launch_tile_lean(const TileArgs& A, cudaStream_t st)
{
    const size_t smem = (size_t)lean_smem_bytes(A.plan);
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute((const void*)k_tile_lean, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    void* args[] = {const_cast<TileArgs*>(&A)};
    return cudaLaunchCooperativeKernel((const void*)k_tile_lean, dim3(A.plan.regions), dim3(kTileThreads), args, smem,
                                       st);
}
