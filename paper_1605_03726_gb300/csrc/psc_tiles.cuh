// psc_tiles.cuh -- owner-computes persistent kernel for stretches of events of
// a species without reactions (part of psc_kernels.cu's translation unit: it
// uses that file's stencil, Philox, mirror and claim helpers).
//
// Each block owns a box of whole mirror bricks (4 x 4 x 2 voxels per word)
// and keeps its vacancy bits, plus one brick of halo around it, in shared
// memory for the whole stretch.  Per event (Sec. 2.3, synchronous rule):
//   claim    every molecule of the box draws its direction; if the target is
//            vacant in the snapshot and no other voxel next to the target is
//            occupied, nobody else can want the target and the hop needs no
//            claim; otherwise the molecule claims the target in the global
//            table (lowest id wins), as the event kernels do;
//   commit   winners and unclaimed hops move: the bits of the box change in
//            shared memory; bits of the box's outermost brick layer (which
//            neighbouring boxes read as halo) also change in the global
//            mirror by atomic XOR; a molecule that leaves the box is appended
//            to the inbox of the box it enters, and joins that box's bucket
//            at the start of the next event.
// Between the phases the blocks meet at the bounded grid barrier.  Only the
// halo refresh, the contested claims, the outer-layer updates and the
// hand-overs touch global memory, instead of a bit read, a claim, a claim
// read-back and a bit update for every molecule.
//
// Where the boxes hold the wrap-around of a periodic axis, the halo copies of
// voxels are refreshed from the global mirror; every voxel has exactly one
// owner (its brick's box), whose shared copy is the one that changes.

__device__ __forceinline__ int tile_cut(int a, int nb, int p) { return (int)(((int64_t)a * nb) / p); }
__device__ __forceinline__ int tile_owner(int b, int nb, int p) { return (int)((((int64_t)b + 1) * p - 1) / nb); }

struct TileBox {
    int bi0, bj0, bk0;         // first brick of the region
    int ei, ej, ek;            // region extent in bricks
    int BI, BJ, BK;            // box extent (region + one brick each side)
    int zoff3;                 // FCC: global k mod 3 = (z + zoff3) mod 3 for box coordinate z; HCP: -1
};

// FCC layer class k mod 3 of box coordinate z (-1 on HCP lattices, known
// at compile time so that the HCP kernel carries no FCC code)
template <bool FCC>
__device__ __forceinline__ int tile_c3(const TileBox& b, int z)
{
    return FCC ? (z + b.zoff3) % 3 : -1;
}

__device__ __forceinline__ TileBox tile_box(const TilePlan& P, int r)
{
    TileBox b;
    const int ri = r % P.pi, rj = (r / P.pi) % P.pj, rk = r / (P.pi * P.pj);
    b.bi0 = tile_cut(ri, P.nbi, P.pi);
    b.bj0 = tile_cut(rj, P.nbj, P.pj);
    b.bk0 = tile_cut(rk, P.nbk, P.pk);
    b.ei = tile_cut(ri + 1, P.nbi, P.pi) - b.bi0;
    b.ej = tile_cut(rj + 1, P.nbj, P.pj) - b.bj0;
    b.ek = tile_cut(rk + 1, P.nbk, P.pk) - b.bk0;
    b.BI = b.ei + 2;
    b.BJ = b.ej + 2;
    b.BK = b.ek + 2;
    b.zoff3 = P.fcc ? ((2 * b.bk0 - 2) % 3 + 3) % 3 : -1;
    return b;
}

// Region of voxel (i, j, k) from the per-axis owner tables in shared memory
// (own[0, nbi) along i, then j, then k; regions per axis < 256).
__device__ __forceinline__ int tile_region_of(const TilePlan& P, const uint8_t* own, int32_t i, int32_t j, int32_t k)
{
    return ((int)own[P.nbi + P.nbj + (k >> 1)] * P.pj + (int)own[P.nbi + (j >> 2)]) * P.pi + (int)own[i >> 2];
}

__device__ __forceinline__ void tile_build_owners(const TilePlan& P, uint8_t* own)
{
    const int total = P.nbi + P.nbj + P.nbk;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
        int a;
        if (b < P.nbi) a = tile_owner(b, P.nbi, P.pi);
        else if (b < P.nbi + P.nbj) a = tile_owner(b - P.nbi, P.nbj, P.pj);
        else a = tile_owner(b - P.nbi - P.nbj, P.nbk, P.pk);
        own[b] = (uint8_t)a;
    }
}

// global mirror word of box word (wx, wy, wz), or -1 outside a reflective wall
__device__ __forceinline__ int64_t tile_global_word(const Geometry& G, const TilePlan& P, const TileBox& b,
                                                    int wx, int wy, int wz)
{
    int gi = b.bi0 - 1 + wx, gj = b.bj0 - 1 + wy, gk = b.bk0 - 1 + wz;
    if (gi < 0 || gi >= P.nbi) {
        if (!(G.bflags & 1u)) return -1;
        gi = gi < 0 ? gi + P.nbi : gi - P.nbi;
    }
    if (gj < 0 || gj >= P.nbj) {
        if (!(G.bflags & 2u)) return -1;
        gj = gj < 0 ? gj + P.nbj : gj - P.nbj;
    }
    if (gk < 0 || gk >= P.nbk) {
        if (!(G.bflags & 4u)) return -1;
        gk = gk < 0 ? gk + P.nbk : gk - P.nbk;
    }
    return ((int64_t)gk * P.nbj + gj) * P.nbi + gi;
}

// Box word index and bit of region voxel (i, j, k) (global coordinates inside the region)
__device__ __forceinline__ void tile_local(const TileBox& b, int32_t i, int32_t j, int32_t k, int& w, uint32_t& m)
{
    w = (((k >> 1) - b.bk0 + 1) * b.BJ + ((j >> 2) - b.bj0 + 1)) * b.BI + ((i >> 2) - b.bi0 + 1);
    m = 1u << (((uint32_t)i & 3u) | (((uint32_t)j & 3u) << 2) | (((uint32_t)k & 1u) << 4));
}

// Is the region voxel (i, j, k) in the region's outermost brick layer (a
// halo brick of some box)?
__device__ __forceinline__ bool tile_outer(const TileBox& b, int32_t i, int32_t j, int32_t k)
{
    const int wx = (i >> 2) - b.bi0, wy = (j >> 2) - b.bj0, wz = (k >> 1) - b.bk0;
    return wx == 0 || wx == b.ei - 1 || wy == 0 || wy == b.ej - 1 || wz == 0 || wz == b.ek - 1;
}

__device__ __forceinline__ FastDiv tile_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d;
    if (d <= 1) { f.m = 0; f.s = -1; return f; }
    int l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned p = 31u + (unsigned)l;
    f.m = (uint32_t)(((1ull << p) + d - 1) / d);
    f.s = (int32_t)(p - 32u);
    return f;
}

// Refresh the halo (every box word outside the region) from the global
// mirror.  Word q of the halo: first the full rows of the outer faces (rows
// with wz = 0 or BK - 1, or wy = 0 or BJ - 1), then the two end words of every
// other row; each thread issues its loads in groups of eight.
__device__ __forceinline__ void tile_refresh_halo(const Geometry& G, const TilePlan& P, const TileBox& b,
                                                  const FastDiv& div_bi, const FastDiv& div_bj2,
                                                  const uint32_t* bits, uint32_t* box)
{
    const int BI = b.BI, BJ = b.BJ, BK = b.BK;
    const int face_rows = 2 * BJ + 2 * (BK - 2);
    const int n_face = face_rows * BI;
    const int total = n_face + 2 * (BJ - 2) * (BK - 2);
    constexpr int H = 8;
    for (int q0 = threadIdx.x; q0 < total; q0 += H * blockDim.x) {
        int idx[H];
        uint32_t val[H];
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int q = q0 + h * blockDim.x;
            idx[h] = -1;
            val[h] = 0u;
            if (q >= total) continue;
            int wx, wy, wz;
            if (q < n_face) {
                const int fr = (int)fdiv((uint32_t)q, div_bi);
                wx = q - fr * BI;
                if (fr < BJ) { wz = 0; wy = fr; }
                else if (fr < 2 * BJ) { wz = BK - 1; wy = fr - BJ; }
                else { const int f2 = fr - 2 * BJ; wz = 1 + (f2 >> 1); wy = (f2 & 1) ? BJ - 1 : 0; }
            } else {
                const int q2 = q - n_face, ir = q2 >> 1;
                const int zz = (int)fdiv((uint32_t)ir, div_bj2);
                wx = (q2 & 1) ? BI - 1 : 0;
                wz = 1 + zz;
                wy = 1 + ir - zz * (BJ - 2);
            }
            const int64_t gw = tile_global_word(G, P, b, wx, wy, wz);
            idx[h] = (wz * BJ + wy) * BI + wx;
            if (gw >= 0) val[h] = __ldcg(&bits[gw]);
        }
#pragma unroll
        for (int h = 0; h < H; ++h)
            if (idx[h] >= 0) box[idx[h]] = val[h];
    }
}

// Claim-phase decision of a molecule: bit 31 it claimed its target, bit 30
// it hops without a claim, bits 24-29 its step (dx + 1) | (dy + 1) << 2 |
// (dz + 1) << 4, so the commit phase needs no second stencil look-up.
constexpr uint32_t kTileClaimed = 0x80000000u;
constexpr uint32_t kTileMove = 0x40000000u;

__device__ __forceinline__ uint32_t tile_pack_step(int dx, int dy, int dz)
{
    return (uint32_t)((dx + 1) | ((dy + 1) << 2) | ((dz + 1) << 4)) << 24;
}

__device__ __forceinline__ void tile_step_of(uint32_t st, int& dx, int& dy, int& dz)
{
    const uint32_t q = st >> 24;
    dx = (int)(q & 3u) - 1;
    dy = (int)((q >> 2) & 3u) - 1;
    dz = (int)((q >> 4) & 3u) - 1;
}

// Molecules in a bucket are stored by their coordinates relative to the
// region's first voxel, x | y << 11 | z << 22 (regions of at most 2048 x 2048
// x 1024 voxels); box coordinates add the halo: (x + 4, y + 4, z + 2).
__device__ __forceinline__ uint32_t tile_pack(int lx, int ly, int lz)
{
    return (uint32_t)lx | ((uint32_t)ly << 11) | ((uint32_t)lz << 22);
}

// Global voxel of box coordinates (x, y, z), wrapped; false behind a
// reflective wall.  *wrap: change of the packed wrap counters.
__device__ __forceinline__ bool tile_global(const Geometry& G, const TileBox& b, int x, int y, int z, int32_t& i,
                                            int32_t& j, int32_t& k, uint64_t& wrap)
{
    i = x - 4 + 4 * b.bi0;
    j = y - 4 + 4 * b.bj0;
    k = z - 2 + 2 * b.bk0;
    wrap = 0;
    if (i < 0) {
        if (!(G.bflags & 1u)) return false;
        i += G.ni; wrap |= 0xFFFFull;
    } else if (i >= G.ni) {
        if (!(G.bflags & 1u)) return false;
        i -= G.ni; wrap |= 0x1ull;
    }
    if (j < 0) {
        if (!(G.bflags & 2u)) return false;
        j += G.nj; wrap |= 0xFFFFull << 16;
    } else if (j >= G.nj) {
        if (!(G.bflags & 2u)) return false;
        j -= G.nj; wrap |= 0x1ull << 16;
    }
    if (k < 0) {
        if (!(G.bflags & 4u)) return false;
        k += G.nk; wrap |= 0xFFFFull << 32;
    } else if (k >= G.nk) {
        if (!(G.bflags & 4u)) return false;
        k -= G.nk; wrap |= 0x1ull << 32;
    }
    return true;
}

// Global mirror word of region word (wx, wy, wz) (box word coordinates, 1..e)
__device__ __forceinline__ int64_t tile_region_word(const TilePlan& P, const TileBox& b, int wx, int wy, int wz)
{
    return ((int64_t)(b.bk0 - 1 + wz) * P.nbj + (b.bj0 - 1 + wy)) * P.nbi + (b.bi0 - 1 + wx);
}

// Stencil offset of direction d for box coordinates (x, y, z) (Sec. 2.1); on
// FCC lattices (App. B) c3 = k mod 3 picks the j offsets and the row parity
// (box and global coordinates share the parities of j and k: the box origin
// is a whole number of bricks away)
__device__ __forceinline__ void tile_step(int d, int y, int z, int c3, int& dx, int& dy, int& dz)
{
    uint32_t wi, wj;
    if (c3 < 0) {
        wi = ((y + z) & 1) ? c_stencil[1] : c_stencil[0];
        wj = (z & 1) ? c_stencil[3] : c_stencil[2];
    } else {
        wi = ((y + (c3 == 1 ? 1 : 0)) & 1) ? c_stencil[1] : c_stencil[0];
        wj = c_stencil[5 + c3];
    }
    dx = (int)((wi >> (2 * d)) & 3u) - 1;
    dy = (int)((wj >> (2 * d)) & 3u) - 1;
    dz = (int)((c_stencil[4] >> (2 * d)) & 3u) - 1;
}

// Neighbourhood masks.  For the 32 places c = (x & 3) | (y & 3) << 2 |
// (z & 1) << 4 of a voxel in its brick word (its bit index), mask[c][q] has
// the bits of the voxel itself and of its 12 neighbours (Sec. 2.1) in the
// eight words q = xb | yb << 1 | zb << 2 around it, counted from the word
// holding (x - 1, y - 1, z - 1).  Only the low bits of (x, y, z) matter: the
// stencil depends on the parities of y + z and z, and the brick steps on x & 3,
// y & 3, z & 1.
__device__ __forceinline__ void tile_build_nbmask(uint32_t* mask, int fcc)
{
    const int entries = fcc ? 96 : 32;          // FCC: one table per layer class k mod 3
    for (int e = threadIdx.x; e < entries * 8; e += blockDim.x) mask[e] = 0u;
    __syncthreads();
    if (threadIdx.x < entries) {
        const int c = threadIdx.x;
        const int c3 = fcc ? (c >> 5) : -1;
        const int x = 4 + (c & 3), y = 4 + ((c >> 2) & 3), z = 2 + ((c >> 4) & 1);
        const int wx0 = (x - 1) >> 2, wy0 = (y - 1) >> 2, wz0 = (z - 1) >> 1;
        for (int d = -1; d < 12; ++d) {
            int dx = 0, dy = 0, dz = 0;
            if (d >= 0) tile_step(d, y, z, c3, dx, dy, dz);
            const int nx = x + dx, ny = y + dy, nz = z + dz;
            const int q = ((nx >> 2) - wx0) | (((ny >> 2) - wy0) << 1) | (((nz >> 1) - wz0) << 2);
            mask[c * 8 + q] |= 1u << ((nx & 3) | ((ny & 3) << 2) | ((nz & 1) << 4));
        }
    }
    __syncthreads();
}

// Occupied voxels among the target (tx, ty, tz) and its 12 neighbours.  One
// of them is the mover, so 1 means: the target is vacant and no other
// molecule can reach it.
__device__ __forceinline__ int tile_nb_count(const uint32_t* box, const uint32_t* nbmask, int BI, int BIJ,
                                             int BJ, int tx, int ty, int tz, int c3)
{
    const int c = ((tx & 3) | ((ty & 3) << 2) | ((tz & 1) << 4)) + (c3 > 0 ? 32 * c3 : 0);
    const int w0 = (((tz - 1) >> 1) * BJ + ((ty - 1) >> 2)) * BI + ((tx - 1) >> 2);
    const uint4 m0 = *reinterpret_cast<const uint4*>(nbmask + c * 8);
    const uint4 m1 = *reinterpret_cast<const uint4*>(nbmask + c * 8 + 4);
    return __popc(box[w0] & m0.x) + __popc(box[w0 + 1] & m0.y) + __popc(box[w0 + BI] & m0.z) +
           __popc(box[w0 + BI + 1] & m0.w) + __popc(box[w0 + BIJ] & m1.x) + __popc(box[w0 + BIJ + 1] & m1.y) +
           __popc(box[w0 + BIJ + BI] & m1.z) + __popc(box[w0 + BIJ + BI + 1] & m1.w);
}

// Move the inbox of region r into bucket buffer `buf` (length n) and set the
// arrivals' bits in the box.
__device__ __forceinline__ void tile_ingest(const TileArgs& A, int r, const TileBox& b, uint32_t* box, int& n,
                                            int buf, int* s_misc)
{
    const int cap = A.plan.cap;
    if (threadIdx.x == 0) s_misc[0] = min(*((volatile int32_t*)&A.in_cnt[r]), cap);
    __syncthreads();
    const int m = s_misc[0];
    const int64_t base = (int64_t)r * cap;
    for (int x = threadIdx.x; x < m; x += blockDim.x) {
        const int32_t t = __ldcg(&A.in_vox[base + x]);
        const uint32_t id = __ldcg(&A.in_ids[base + x]);
        int32_t i, j, k;
        decode(A.ev.geo, (uint32_t)t, i, j, k);
        int w;
        uint32_t mk;
        tile_local(b, i, j, k, w, mk);
        atomicOr(&box[w], mk);
        if (n + x < cap) {
            A.b_vox[buf][base + n + x] = (int32_t)tile_pack(i - 4 * b.bi0, j - 4 * b.bj0, k - 2 * b.bk0);
            A.b_ids[buf][base + n + x] = id;
        } else {
            atomicOr(&A.ev.sc->err, kErrListOverflow);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) A.in_cnt[r] = 0;
    n = min(n + m, cap);
}

// Wait until every box next to region r (up to 26, across periodic wraps)
// has published flags[q] >= target.  Bounded like the grid barrier; false
// (error raised) on time-out.  A nonzero barrier_phantom (tests of the
// time-out path) raises the target beyond anything published.
__device__ __forceinline__ bool tile_wait_neighbours(const TileArgs& A, const uint32_t* flags, int r,
                                                     uint32_t target, int* s_flag)
{
    const TilePlan& P = A.plan;
    const uint32_t bf = A.ev.geo.bflags;
    target += A.barrier_phantom ? 0x40000000u : 0u;
    if (threadIdx.x == 0) *s_flag = 1;
    __syncthreads();
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
                        *s_flag = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *s_flag != 0;
}

// Shared-memory areas of the tile kernel, after the box.
struct TileShared {
    uint32_t* box;
    uint32_t* nbmask;          // [32][8], FCC [3][32][8]
    int32_t* o_t;              // outbox: departures of an event
    uint32_t* o_id;
    int32_t* o_q;
    int32_t* queue;            // bucket slots whose handling is deferred
    uint8_t* own;              // owner tables
};

__device__ __forceinline__ TileShared tile_shared(uint32_t* smem, const TilePlan& P)
{
    TileShared S;
    S.box = smem;
    S.nbmask = smem + ((P.box_words + 3) & ~3);
    S.o_t = reinterpret_cast<int32_t*>(S.nbmask + (P.fcc ? 96 : 32) * 8);
    S.o_id = reinterpret_cast<uint32_t*>(S.o_t + kTileOutbox);
    S.o_q = S.o_t + 2 * kTileOutbox;
    S.queue = S.o_t + 3 * kTileOutbox;
    S.own = reinterpret_cast<uint8_t*>(S.queue + kTileQueue);
    return S;
}

// Box coordinates of a molecule from its packed region coordinates
__device__ __forceinline__ void tile_unpack(uint32_t w, int& x, int& y, int& z)
{
    x = (int)(w & 0x7FFu) + 4;
    y = (int)((w >> 11) & 0x7FFu) + 4;
    z = (int)(w >> 22) + 2;
}

// A molecule of the box (packed coordinates w) takes the step its decision
// st holds (it won the target or needed no claim).  Updates the box and the
// global mirror's outer layer, hands it over if it leaves the box; returns
// whether it stays and, if so, its new packed coordinates.
__device__ __forceinline__ bool tile_apply_move(const TileArgs& A, const TileBox& b, const TileShared& S, int r,
                                                int* s_out_n, uint32_t w, uint32_t id, uint32_t st, uint32_t& neww)
{
    const Geometry& G = A.ev.geo;
    int x, y, z, dx, dy, dz;
    tile_unpack(w, x, y, z);
    tile_step_of(st, dx, dy, dz);
    const int tx = x + dx, ty = y + dy, tz = z + dz;
    const int vwx = x >> 2, vwy = y >> 2, vwz = z >> 1;
    const int wv = (vwz * b.BJ + vwy) * b.BI + vwx;
    const uint32_t mv = 1u << ((x & 3) | ((y & 3) << 2) | ((z & 1) << 4));
    const bool v_outer = vwx == 1 || vwx == b.ei || vwy == 1 || vwy == b.ej || vwz == 1 || vwz == b.ek;
    int lx = tx - 4, ly = ty - 4, lz = tz - 2;               // target relative to the region
    bool in_region = tx >= 4 && tx < 4 + 4 * b.ei && ty >= 4 && ty < 4 + 4 * b.ej && tz >= 2 && tz < 2 + 2 * b.ek;
    int32_t gi = 0, gj = 0, gk = 0;
    if (!in_region) {
        uint64_t wr;
        tile_global(G, b, tx, ty, tz, gi, gj, gk, wr);
        if (wr) {
            uint64_t* wp = &A.img_id[id - A.id_lo];
            *wp = img_add(*wp, wr);
        }
        if (tile_region_of(A.plan, S.own, gi, gj, gk) == r) {
            // the region wraps around onto itself along a periodic axis
            lx = gi - 4 * b.bi0;
            ly = gj - 4 * b.bj0;
            lz = gk - 2 * b.bk0;
            in_region = true;
        }
    }
    if (in_region) {
        const int twx = (lx >> 2) + 1, twy = (ly >> 2) + 1, twz = (lz >> 1) + 1;
        const int wt = (twz * b.BJ + twy) * b.BI + twx;
        const uint32_t mt = 1u << ((lx & 3) | ((ly & 3) << 2) | ((lz & 1) << 4));
        if (wv == wt) {
            atomicXor(&S.box[wv], mv | mt);
        } else {
            atomicXor(&S.box[wv], mv);
            atomicXor(&S.box[wt], mt);
        }
        const bool t_outer = twx == 1 || twx == b.ei || twy == 1 || twy == b.ej || twz == 1 || twz == b.ek;
        if (v_outer && t_outer && wv == wt) {
            atomicXor(&A.ev.bits[tile_region_word(A.plan, b, vwx, vwy, vwz)], mv | mt);
        } else {
            if (v_outer) atomicXor(&A.ev.bits[tile_region_word(A.plan, b, vwx, vwy, vwz)], mv);
            if (t_outer) atomicXor(&A.ev.bits[tile_region_word(A.plan, b, twx, twy, twz)], mt);
        }
        neww = tile_pack(lx, ly, lz);
        return true;
    }
    // into another box: hand the molecule over (through the outbox)
    atomicXor(&S.box[wv], mv);
    atomicXor(&A.ev.bits[tile_region_word(A.plan, b, vwx, vwy, vwz)], mv);
    const BitPos gt = bitpos(G, gi, gj, gk);
    atomicXor(&A.ev.bits[gt.word], gt.mask);
    const int q = tile_region_of(A.plan, S.own, gi, gj, gk);
    const int32_t t = gi + G.ni * (gj + G.nj * gk);
    const int o = atomicAdd(s_out_n, 1);
    if (o < kTileOutbox) {
        S.o_t[o] = t;
        S.o_id[o] = id;
        S.o_q[o] = q;
    } else {
        const int cap = A.plan.cap;
        const int slot = atomicAdd(&A.in_cnt[q], 1);
        if (slot < cap) {
            A.in_vox[(int64_t)q * cap + slot] = t;
            A.in_ids[(int64_t)q * cap + slot] = id;
        } else {
            atomicOr(&A.ev.sc->err, kErrListOverflow);
        }
    }
    return false;
}

// Keep a survivor: one shared-memory atomic per warp reserves the warp's slots
// in the other bucket buffer.  Called by all lanes.
__device__ __forceinline__ void tile_keep(bool keep, uint32_t w, uint32_t id, int* s_keep_n, int32_t* ov, uint32_t* oi)
{
    const int lane = threadIdx.x & 31;
    const unsigned ball = __ballot_sync(0xFFFFFFFFu, keep);
    int wbase = 0;
    if (lane == 0 && ball) wbase = atomicAdd(s_keep_n, __popc(ball));
    wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
    if (keep) {
        const int o = wbase + __popc(ball & ((1u << lane) - 1u));
        ov[o] = (int32_t)w;
        oi[o] = id;
    }
}

// Global voxel of the target of a molecule (packed w, decision st)
__device__ __forceinline__ void tile_target_global(const Geometry& G, const TileBox& b, uint32_t w, uint32_t st,
                                                   Nb& nb)
{
    int x, y, z, dx, dy, dz;
    tile_unpack(w, x, y, z);
    tile_step_of(st, dx, dy, dz);
    tile_global(G, b, x + dx, y + dy, z + dz, nb.i, nb.j, nb.k, nb.wrap);
    nb.t = nb.i + G.ni * (nb.j + G.nj * nb.k);
}

// Publish that region r has finished a phase of the event (flags[r] = value)
__device__ __forceinline__ void tile_publish(uint32_t* flags, int r, uint32_t value)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(&flags[r], value);
    }
}

template <bool FCC>
__global__ void __launch_bounds__(kTileThreads, kTileBlocksPerSM) k_tile_run(const TileArgs A)
{
    extern __shared__ uint32_t smem[];
    // s_misc: arrivals, survivors, outbox entries, wait flag, -, commit queue
    __shared__ int s_misc[6];
    const EventArgs& a = A.ev;
    const Geometry& G = a.geo;
    const int r = blockIdx.x;
    const TileBox b = tile_box(A.plan, r);
    const TileShared S = tile_shared(smem, A.plan);
    uint32_t* box = S.box;
    const int nbox = b.BI * b.BJ * b.BK;
    const int BIJ = b.BI * b.BJ;
    const int cap = A.plan.cap;
    const int64_t base = (int64_t)r * cap;
    const uint32_t c2 = ((uint32_t)a.s << 4) | kTagEvent;
    uint32_t* claim = A.claim;
    constexpr int U = 2;                                 // molecules whose memory operations go out together
    // box coordinates of the lattice along reflective axes (targets outside are walls)
    const int xlo = (G.bflags & 1u) ? INT_MIN : 4 - 4 * b.bi0, xhi = (G.bflags & 1u) ? INT_MAX : xlo + G.ni;
    const int ylo = (G.bflags & 2u) ? INT_MIN : 4 - 4 * b.bj0, yhi = (G.bflags & 2u) ? INT_MAX : ylo + G.nj;
    const int zlo = (G.bflags & 4u) ? INT_MIN : 2 - 2 * b.bk0, zhi = (G.bflags & 4u) ? INT_MAX : zlo + G.nk;
    const int rx1 = 4 + 4 * b.ei, ry1 = 4 + 4 * b.ej, rz1 = 2 + 2 * b.ek;   // region: [4, rx1) x [4, ry1) x [2, rz1)
    const FastDiv div_bi = tile_fastdiv((uint32_t)b.BI), div_bj2 = tile_fastdiv((uint32_t)(b.BJ - 2));
    tile_build_owners(A.plan, S.own);
    tile_build_nbmask(S.nbmask, A.plan.fcc);
    // region and halo bits from the global mirror
    for (int q = threadIdx.x; q < nbox; q += blockDim.x) {
        const int wx = q % b.BI, wy = (q / b.BI) % b.BJ, wz = q / (b.BI * b.BJ);
        const int64_t gw = tile_global_word(G, A.plan, b, wx, wy, wz);
        box[q] = gw >= 0 ? __ldcg(&a.bits[gw]) : 0u;
    }
    int n = *((volatile int32_t*)&A.b_cnt[r]);
    // the scatter left voxel indices: store coordinates relative to the region
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        int32_t i, j, k;
        decode(G, (uint32_t)A.b_vox[0][base + x], i, j, k);
        A.b_vox[0][base + x] = (int32_t)tile_pack(i - 4 * b.bi0, j - 4 * b.bj0, k - 2 * b.bk0);
    }
    unsigned long long n_att = 0, n_hop = 0;
    __syncthreads();
    for (int e = 0; e < A.n_events; ++e) {
        const uint32_t g = a.g + (uint32_t)e;
        const int cur = e & 1;
        const int32_t* bv = A.b_vox[cur] + base;
        const uint32_t* bi = A.b_ids[cur] + base;
        uint32_t* bs = A.b_state + base;
        if (e > 0) {
            // the neighbours' last commits: halo bits, arrivals, reset claim words
            if (A.nbr_sync && !tile_wait_neighbours(A, A.done, r, (uint32_t)e, &s_misc[3])) return;
            tile_ingest(A, r, b, box, n, cur, s_misc);
            tile_refresh_halo(G, A.plan, b, div_bi, div_bj2, a.bits, box);
            __syncthreads();
        }
        // ---- claim phase ----
        for (int c0 = 0; c0 < n; c0 += U * blockDim.x) {
            uint32_t vv[U], ii[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int x = c0 + u * blockDim.x + threadIdx.x;
                vv[u] = x < n ? (uint32_t)__ldcg(bv + x) : 0u;
                ii[u] = x < n ? __ldcg(bi + x) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int xm = c0 + u * blockDim.x + threadIdx.x;
                if (xm >= n) continue;
                int x, y, z, dx, dy, dz;
                tile_unpack(vv[u], x, y, z);
                uint32_t rnd[4];
                philox(ii[u], g, c2, 0u, a.key0, a.key1, rnd);
                const int d = (int)__umulhi(rnd[0], 12u);
                tile_step(d, y, z, tile_c3<FCC>(b, z), dx, dy, dz);
                uint32_t st = tile_pack_step(dx, dy, dz);
                const int tx = x + dx, ty = y + dy, tz = z + dz;
                if (tx >= xlo && tx < xhi && ty >= ylo && ty < yhi && tz >= zlo && tz < zhi) {
                    if (tile_nb_count(box, S.nbmask, b.BI, BIJ, b.BJ, tx, ty, tz, tile_c3<FCC>(b, tz)) == 1) {
                        st |= kTileMove;                 // only the mover itself is next to the target
                    } else if (!(box[((tz >> 1) * b.BJ + (ty >> 2)) * b.BI + (tx >> 2)] &
                                 (1u << ((tx & 3) | ((ty & 3) << 2) | ((tz & 1) << 4))))) {
                        // vacant, but other molecules can reach it: the lowest id wins
                        int32_t i, j, k;
                        uint64_t w;
                        tile_global(G, b, tx, ty, tz, i, j, k, w);
                        atomicMin(&claim[i + G.ni * (j + G.nj * k)], ii[u]);
                        st |= kTileClaimed;
                    }
                }
                bs[xm] = st;
            }
        }
        n_att += (unsigned long long)n;
        if (threadIdx.x == 0) {
            s_misc[1] = 0;
            s_misc[2] = 0;
            s_misc[5] = 0;
        }
        if (A.nbr_sync) {
            // a claim word is touched only by boxes that are all neighbours of each other
            tile_publish(A.claimed, r, (uint32_t)(e + 1));
            if (!tile_wait_neighbours(A, A.claimed, r, (uint32_t)(e + 1), &s_misc[3])) return;
        } else if (!grid_barrier(A.barrier, &a.sc->err, A.barrier_timeout_ns, A.barrier_phantom)) {
            return;
        }
        // ---- commit phase: hops inside the box here, everything else queued ----
        int32_t* ov = A.b_vox[cur ^ 1] + base;
        uint32_t* oi = A.b_ids[cur ^ 1] + base;
        for (int c0 = 0; c0 < n; c0 += U * blockDim.x) {
            uint32_t vv[U], ii[U], ss[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int x = c0 + u * blockDim.x + threadIdx.x;
                vv[u] = x < n ? (uint32_t)__ldcg(bv + x) : 0u;
                ii[u] = x < n ? __ldcg(bi + x) : 0u;
                ss[u] = x < n ? __ldcg(bs + x) : 0u;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int xm = c0 + u * blockDim.x + threadIdx.x;
                const uint32_t st = ss[u];
                uint32_t w = vv[u];
                bool keep = xm < n;
                bool defer = (st & kTileClaimed) != 0u;
                if (st & kTileMove) {
                    int x, y, z, dx, dy, dz;
                    tile_unpack(w, x, y, z);
                    tile_step_of(st, dx, dy, dz);
                    const int tx = x + dx, ty = y + dy, tz = z + dz;
                    if (tx >= 4 && tx < rx1 && ty >= 4 && ty < ry1 && tz >= 2 && tz < rz1) {
                        uint32_t neww;
                        tile_apply_move(A, b, S, r, &s_misc[2], w, ii[u], st, neww);
                        w = neww;
                        ++n_hop;
                    } else {
                        defer = true;
                    }
                }
                if (defer) {
                    const int k = atomicAdd(&s_misc[5], 1);
                    if (k < kTileQueue) {
                        S.queue[k] = xm;
                        keep = false;
                    } else {
                        // queue full: handle it here
                        bool win = (st & kTileMove) != 0u;
                        if (!win) {
                            Nb nb;
                            tile_target_global(G, b, w, st, nb);
                            win = __ldcg(&claim[nb.t]) == ii[u];
                            if (win) claim[nb.t] = kNoClaim;
                        }
                        if (win) {
                            uint32_t neww = w;
                            keep = tile_apply_move(A, b, S, r, &s_misc[2], w, ii[u], st, neww);
                            w = neww;
                            ++n_hop;
                        }
                    }
                }
                tile_keep(keep, w, ii[u], &s_misc[1], ov, oi);
            }
        }
        __syncthreads();
        {
            // queued molecules: claim read-backs of a batch in flight together
            const int m = min(s_misc[5], kTileQueue);
            for (int c0 = 0; c0 < m; c0 += U * blockDim.x) {
                int32_t xx[U], tt[U];
                uint32_t vv[U], ii[U], ss[U], rb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int k = c0 + u * blockDim.x + threadIdx.x;
                    xx[u] = k < m ? S.queue[k] : -1;
                    vv[u] = xx[u] >= 0 ? (uint32_t)__ldcg(bv + xx[u]) : 0u;
                    ii[u] = xx[u] >= 0 ? __ldcg(bi + xx[u]) : 0u;
                    ss[u] = xx[u] >= 0 ? __ldcg(bs + xx[u]) : 0u;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    rb[u] = 0u;
                    tt[u] = -1;
                    if (!(ss[u] & kTileClaimed)) continue;
                    Nb nb;
                    tile_target_global(G, b, vv[u], ss[u], nb);
                    tt[u] = nb.t;
                    rb[u] = __ldcg(&claim[nb.t]);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t st = ss[u];
                    uint32_t w = vv[u];
                    bool keep = xx[u] >= 0;
                    bool win = (st & kTileMove) != 0u;
                    if ((st & kTileClaimed) && rb[u] == ii[u]) {
                        win = true;
                        claim[tt[u]] = kNoClaim;         // the winner resets the word
                    }
                    if (keep && win) {
                        uint32_t neww = w;
                        keep = tile_apply_move(A, b, S, r, &s_misc[2], w, ii[u], st, neww);
                        w = neww;
                        ++n_hop;
                    }
                    tile_keep(keep, w, ii[u], &s_misc[1], ov, oi);
                }
            }
        }
        __syncthreads();
        n = s_misc[1];
        // the outbox to the inboxes of the boxes the molecules entered
        {
            const int m = min(s_misc[2], kTileOutbox);
            for (int o = threadIdx.x; o < m; o += blockDim.x) {
                const int q = S.o_q[o];
                const int slot = atomicAdd(&A.in_cnt[q], 1);
                if (slot < cap) {
                    A.in_vox[(int64_t)q * cap + slot] = S.o_t[o];
                    A.in_ids[(int64_t)q * cap + slot] = S.o_id[o];
                } else {
                    atomicOr(&a.sc->err, kErrListOverflow);
                }
            }
        }
        if (A.nbr_sync) {
            tile_publish(A.done, r, (uint32_t)(e + 1));
        } else if (!grid_barrier(A.barrier, &a.sc->err, A.barrier_timeout_ns, A.barrier_phantom)) {
            return;
        }
    }
    // the last event's arrivals, then the region's bits back to the mirror
    if (A.n_events > 0 && A.nbr_sync && !tile_wait_neighbours(A, A.done, r, (uint32_t)A.n_events, &s_misc[3]))
        return;
    if (A.n_events > 0) tile_ingest(A, r, b, box, n, A.n_events & 1, s_misc);
    __syncthreads();
    for (int q = threadIdx.x; q < b.ei * b.ej * b.ek; q += blockDim.x) {
        const int wx = 1 + q % b.ei, wy = 1 + (q / b.ei) % b.ej, wz = 1 + q / (b.ei * b.ej);
        a.bits[tile_region_word(A.plan, b, wx, wy, wz)] = box[(wz * b.BJ + wy) * b.BI + wx];
    }
    if (threadIdx.x == 0) A.b_cnt[r] = n;
    if (a.collect_stats) {
        if (threadIdx.x == 0) atomicAdd(&a.sc->stats[kStatAttempts], n_att);
        flush_stat(&a.sc->stats[kStatHops], n_hop);
    }
}

// list -> buckets: a block histograms its molecules by region in shared
// memory, reserves each region's range with one atomic, then writes
__global__ void __launch_bounds__(1024) k_tile_scatter(const TileArgs A)
{
    extern __shared__ int s_hist[];                      // [2 * regions] + owner tables
    const EventArgs& a = A.ev;
    const int R = A.plan.regions;
    uint8_t* own = reinterpret_cast<uint8_t*>(s_hist + 2 * R);
    const int n = *a.count;
    tile_build_owners(A.plan, own);
    for (int q = threadIdx.x; q < R; q += blockDim.x) s_hist[q] = 0;
    __syncthreads();
    const int per_block = (n + gridDim.x - 1) / gridDim.x;
    const int lo = blockIdx.x * per_block, hi = min(n, lo + per_block);
    constexpr int kPer = 8;
    int reg[kPer], rank[kPer];
    for (int c0 = lo; c0 < hi; c0 += blockDim.x * kPer) {
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int x = c0 + u * blockDim.x + threadIdx.x;
            reg[u] = -1;
            if (x < hi) {
                int32_t i, j, k;
                decode(a.geo, (uint32_t)a.list.vox[x], i, j, k);
                reg[u] = tile_region_of(A.plan, own, i, j, k);
                rank[u] = atomicAdd(&s_hist[reg[u]], 1);
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < R; q += blockDim.x) {
            const int c = s_hist[q];
            s_hist[R + q] = c ? atomicAdd(&A.b_cnt[q], c) : 0;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int x = c0 + u * blockDim.x + threadIdx.x;
            if (reg[u] < 0) continue;
            const int slot = s_hist[R + reg[u]] + rank[u];
            const uint32_t id = a.list.ids[x];
            if (slot < A.plan.cap) {
                A.b_vox[0][(int64_t)reg[u] * A.plan.cap + slot] = a.list.vox[x];
                A.b_ids[0][(int64_t)reg[u] * A.plan.cap + slot] = id;
            } else {
                atomicOr(&a.sc->err, kErrListOverflow);
            }
            A.img_id[id - A.id_lo] = a.list.img[x];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < R; q += blockDim.x) s_hist[q] = 0;
        __syncthreads();
    }
}

// buckets -> list (region after region), wrap counters from the id table;
// the molecules are in the buffer the last event left them in
__global__ void __launch_bounds__(256) k_tile_gather(const TileArgs A)
{
    const EventArgs& a = A.ev;
    const int r = blockIdx.x;
    const int buf = A.n_events & 1;
    __shared__ int s_off;
    if (threadIdx.x == 0) {
        int off = 0;
        for (int q = 0; q < r; ++q) off += min(A.b_cnt[q], A.plan.cap);
        s_off = off;
    }
    __syncthreads();
    const int m = min(A.b_cnt[r], A.plan.cap);
    const int64_t base = (int64_t)r * A.plan.cap;
    const TileBox b = tile_box(A.plan, r);
    for (int x = threadIdx.x; x < m; x += blockDim.x) {
        const int dst = s_off + x;
        if (dst >= a.list.cap) break;
        const uint32_t id = A.b_ids[buf][base + x];
        const uint32_t w = (uint32_t)A.b_vox[buf][base + x];
        const int32_t i = (int32_t)(w & 0x7FFu) + 4 * b.bi0, j = (int32_t)((w >> 11) & 0x7FFu) + 4 * b.bj0,
                      k = (int32_t)(w >> 22) + 2 * b.bk0;
        a.list.vox[dst] = i + a.geo.ni * (j + a.geo.nj * k);
        a.list.ids[dst] = id;
        a.list.img[dst] = A.img_id[id - A.id_lo];
    }
}

int tile_smem_limit(int device)
{
    int optin = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess)
        return 0;
    // kTileBlocksPerSM blocks share an SM; each also reserves 1 KB, plus static shared memory and slack
    const int share = per_sm / kTileBlocksPerSM - 2048;
    return optin - 1024 < share ? optin - 1024 : share;
}

// molecules per region (counts[regions], zeroed by the caller): the loads the
// plan would give the blocks
__global__ void __launch_bounds__(1024) k_tile_count(const TileArgs A, int32_t* counts)
{
    extern __shared__ int s_hist[];                      // [regions] + owner tables
    const EventArgs& a = A.ev;
    const int R = A.plan.regions;
    uint8_t* own = reinterpret_cast<uint8_t*>(s_hist + R);
    const int n = *a.count;
    tile_build_owners(A.plan, own);
    for (int q = threadIdx.x; q < R; q += blockDim.x) s_hist[q] = 0;
    __syncthreads();
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        int32_t i, j, k;
        decode(a.geo, (uint32_t)a.list.vox[x], i, j, k);
        atomicAdd(&s_hist[tile_region_of(A.plan, own, i, j, k)], 1);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < R; q += blockDim.x)
        if (s_hist[q]) atomicAdd(&counts[q], s_hist[q]);
}

void launch_tile_count(const TileArgs& A, int32_t* counts, int blocks, cudaStream_t st)
{
    const int smem = A.plan.regions * (int)sizeof(int) + ((A.plan.nbi + A.plan.nbj + A.plan.nbk + 15) & ~15);
    static int configured = 48 * 1024;
    if (smem > configured) {
        cudaFuncSetAttribute(k_tile_count, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        configured = smem;
    }
    k_tile_count<<<blocks, 1024, smem, st>>>(A, counts);
}

void launch_tile_scatter(const TileArgs& A, int blocks, cudaStream_t st)
{
    const int smem = 2 * A.plan.regions * (int)sizeof(int) + ((A.plan.nbi + A.plan.nbj + A.plan.nbk + 15) & ~15);
    static int configured = 48 * 1024;
    if (smem > configured) {
        cudaFuncSetAttribute(k_tile_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        configured = smem;
    }
    k_tile_scatter<<<blocks, 1024, smem, st>>>(A);
}

template <bool FCC>
static cudaError_t launch_tile_run_t(const TileArgs& A, cudaStream_t st)
{
    const size_t smem = (size_t)tile_smem_bytes(A.plan);
    static size_t configured = 0;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute((const void*)k_tile_run<FCC>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    void* args[] = {const_cast<TileArgs*>(&A)};
    return cudaLaunchCooperativeKernel((const void*)k_tile_run<FCC>, dim3(A.plan.regions), dim3(kTileThreads), args,
                                       smem, st);
}

#include "psc_tiles_lean.cuh"

cudaError_t launch_tile_run(const TileArgs& A, cudaStream_t st)
{
    if (A.plan.lean) return launch_tile_lean(A, st);
    return A.plan.fcc ? launch_tile_run_t<true>(A, st) : launch_tile_run_t<false>(A, st);
}

void launch_tile_gather(const TileArgs& A, cudaStream_t st)
{
    k_tile_gather<<<A.plan.regions, 256, 0, st>>>(A);
}
