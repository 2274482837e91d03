// psc_slab.cuh -- slab decomposition of the lattice along k (part of
// psc_kernels.cu's translation unit: it uses that file's stencil and Philox).
//
// The paper splits the lattice into sub-domains, one per process, each with a
// layer of ghost voxels that is refreshed from the neighbouring sub-domains
// (Sec. 2.5).  Here a slab owns the layers k0 .. k0 + m - 1 of the lattice and
// keeps two ghost layers, one on each side: local layer L = k - k0 + 1, owned
// layers 1 .. m, ghost layers 0 and m + 1.  An event of a species without
// reactions (Sec. 2.3, synchronous rule) takes three steps with an exchange
// with both neighbouring slabs after the first two:
//   claim    every molecule draws its direction; a vacant target is claimed
//            in a per-voxel word (lowest id wins).  The claim words of layers
//            0, 1 and m, m + 1 go to the neighbours, since a target in them
//            can be wanted from both sides;
//   commit   the neighbours' claims are merged (minimum), winners move; a
//            molecule that enters a ghost layer leaves the slab and goes into
//            the message for that neighbour, with the owned boundary layer's
//            bits (layer 1 down, layer m up);
//   apply    the ghost layers take the neighbours' boundary bits (plus the bits
//            of this slab's own departures, which the neighbour had not yet
//            placed), the arrivals join the list.
// Claims of a voxel in layers 2 .. m - 1 come from this slab only, and their
// winner empties the word; the words of layers 0, 1, m, m + 1 are emptied after
// every commit.

constexpr uint8_t kSlabNone = 0xFFu;
constexpr uint8_t kSlabClaimed = 0x80u;

// a commit message: int32 count, int32 pad, entries [tcap], boundary layer bits [lw]
__host__ __device__ __forceinline__ size_t slab_msg_entries_off() { return 8; }
__host__ __device__ __forceinline__ size_t slab_msg_bits_off(int32_t tcap) { return 8 + (size_t)tcap * sizeof(SlabEntry); }

__device__ __forceinline__ bool slab_bit(const SlabArgs& A, int i, int j, int L)
{
    const uint32_t b = (uint32_t)i + (uint32_t)A.ni * (uint32_t)j;
    return (A.bits[(size_t)L * A.lw + (b >> 5)] >> (b & 31u)) & 1u;
}

__device__ __forceinline__ void slab_flip(const SlabArgs& A, int i, int j, int L)
{
    const uint32_t b = (uint32_t)i + (uint32_t)A.ni * (uint32_t)j;
    atomicXor(&A.bits[(size_t)L * A.lw + (b >> 5)], 1u << (b & 31u));
}

__device__ __forceinline__ void slab_set(const SlabArgs& A, int i, int j, int L)
{
    const uint32_t b = (uint32_t)i + (uint32_t)A.ni * (uint32_t)j;
    atomicOr(&A.bits[(size_t)L * A.lw + (b >> 5)], 1u << (b & 31u));
}

// Target of a molecule at local (i, j, L) in direction d (Sec. 2.1 stencil,
// parities of the global j + k and k); false behind a wall along i or j.
// Along k the target is a local layer L - 1 .. L + 1, always inside the array
// (ghost layers behind a reflective wall are all ones).  wrap: the change of
// the packed wrap counters, k included when the step crosses the periodic
// seam of k.
__device__ __forceinline__ bool slab_target(const SlabArgs& A, int i, int j, int L, int d, int& ti, int& tj,
                                            int& tL, uint64_t& wrap)
{
    const int k = A.k0 - 1 + L;                          // global layer of the molecule (owned: inside 0 .. nk-1)
    const uint32_t wi = ((j + k) & 1) ? c_stencil[1] : c_stencil[0];
    const uint32_t wj = (k & 1) ? c_stencil[3] : c_stencil[2];
    const int dk = (int)((c_stencil[4] >> (2 * d)) & 3u) - 1;
    ti = i + (int)((wi >> (2 * d)) & 3u) - 1;
    tj = j + (int)((wj >> (2 * d)) & 3u) - 1;
    tL = L + dk;
    wrap = 0;
    if (ti < 0) {
        if (!(A.bflags & 1u)) return false;
        ti += A.ni; wrap |= 0xFFFFull;
    } else if (ti >= A.ni) {
        if (!(A.bflags & 1u)) return false;
        ti -= A.ni; wrap |= 0x1ull;
    }
    if (tj < 0) {
        if (!(A.bflags & 2u)) return false;
        tj += A.nj; wrap |= 0xFFFFull << 16;
    } else if (tj >= A.nj) {
        if (!(A.bflags & 2u)) return false;
        tj -= A.nj; wrap |= 0x1ull << 16;
    }
    const int tk = k + dk;
    if (tk < 0) wrap |= 0xFFFFull << 32;                  // periodic seam (a wall reads as occupied)
    else if (tk >= A.nk) wrap |= 0x1ull << 32;
    return true;
}

__global__ void k_slab_claim(const SlabArgs A)
{
    const int n = A.count[A.cur];
    const uint32_t c2 = (A.s << 4) | kTagEvent;
    const int32_t* vox = A.vox[A.cur];
    const uint32_t* ids = A.ids[A.cur];
    const uint32_t nij = (uint32_t)A.ni * (uint32_t)A.nj;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t v = (uint32_t)vox[x], id = ids[x];
        const int L = (int)(v / nij), r = (int)(v - (uint32_t)L * nij);
        const int j = r / A.ni, i = r - j * A.ni;
        uint32_t u[4];
        philox(id, A.g, c2, 0u, A.key0, A.key1, u);
        const int d = (int)__umulhi(u[0], 12u);
        int ti, tj, tL;
        uint64_t wrap;
        uint8_t dec = kSlabNone;
        if (slab_target(A, i, j, L, d, ti, tj, tL, wrap) && !slab_bit(A, ti, tj, tL)) {
            atomicMin(&A.claim[(size_t)tL * nij + (uint32_t)ti + (uint32_t)A.ni * (uint32_t)tj], id);
            dec = (uint8_t)(kSlabClaimed | d);
        }
        A.dec[x] = dec;
    }
}

// the neighbours' claims on layers 0, 1 (from below) and m, m + 1 (from above)
__global__ void k_slab_merge(const SlabArgs A)
{
    const uint32_t nij = (uint32_t)A.ni * (uint32_t)A.nj;
    const size_t per = 2 * (size_t)nij;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < 2 * per; q += (size_t)gridDim.x * blockDim.x) {
        const int side = q >= per ? 1 : 0;
        const size_t w = q - side * per;
        if (!A.has[side]) continue;
        const size_t dst = side == 0 ? w : (size_t)A.m * nij + w;
        const uint32_t o = A.recv_claim[side][w];
        if (o < A.claim[dst]) A.claim[dst] = o;
    }
}

// commit: winners move; survivors go to the other list buffer, molecules
// entering a ghost layer to the message for that side
__global__ void k_slab_commit(const SlabArgs A)
{
    const int n = A.count[A.cur];
    const int nxt = A.cur ^ 1;
    const int32_t* vox = A.vox[A.cur];
    const uint32_t* ids = A.ids[A.cur];
    const uint64_t* img = A.img[A.cur];
    const uint32_t nij = (uint32_t)A.ni * (uint32_t)A.nj;
    const int lane = threadIdx.x & 31;
    for (int x0 = blockIdx.x * blockDim.x; x0 < n; x0 += gridDim.x * blockDim.x) {
        const int x = x0 + threadIdx.x;
        bool keep = x < n;
        uint32_t v = 0, id = 0;
        uint64_t w = 0;
        if (keep) {
            v = (uint32_t)vox[x];
            id = ids[x];
            w = img[x];
            const uint8_t dec = A.dec[x];
            if (dec != kSlabNone) {
                const int L = (int)(v / nij), r = (int)(v - (uint32_t)L * nij);
                const int j = r / A.ni, i = r - j * A.ni;
                int ti, tj, tL;
                uint64_t wrap;
                slab_target(A, i, j, L, dec & 0x0F, ti, tj, tL, wrap);
                const size_t cw = (size_t)tL * nij + (uint32_t)ti + (uint32_t)A.ni * (uint32_t)tj;
                if (A.claim[cw] == id) {
                    if (tL >= 2 && tL <= A.m - 1) A.claim[cw] = kNoClaim;   // boundary layers are emptied in full
                    slab_flip(A, i, j, L);
                    slab_set(A, ti, tj, tL);
                    w = img_add(w, wrap);
                    v = (uint32_t)ti + (uint32_t)A.ni * ((uint32_t)tj + (uint32_t)A.nj * (uint32_t)tL);
                    if (tL == 0 || tL == A.m + 1) {
                        const int side = tL == 0 ? 0 : 1;
                        uint8_t* msg = A.send_commit[side];
                        const int slot = atomicAdd(reinterpret_cast<int32_t*>(msg), 1);
                        if (slot < A.tcap) {
                            SlabEntry* e = reinterpret_cast<SlabEntry*>(msg + slab_msg_entries_off()) + slot;
                            int tk = A.k0 - 1 + tL;
                            if (tk < 0) tk += A.nk;
                            else if (tk >= A.nk) tk -= A.nk;
                            e->i = ti; e->j = tj; e->k = tk; e->id = id; e->img = w;
                        } else {
                            atomicOr(A.err, kErrListOverflow);
                        }
                        keep = false;
                    }
                }
            }
        }
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, keep);
        int wbase = 0;
        if (lane == 0 && ball) wbase = atomicAdd(&A.count[nxt], __popc(ball));
        wbase = __shfl_sync(0xFFFFFFFFu, wbase, 0);
        if (keep) {
            const int o = wbase + __popc(ball & ((1u << lane) - 1u));
            if (o < A.cap) {
                A.vox[nxt][o] = (int32_t)v;
                A.ids[nxt][o] = id;
                A.img[nxt][o] = w;
            } else {
                atomicOr(A.err, kErrListOverflow);
            }
        }
    }
}

// after the commit: the owned boundary layers' bits into the messages, the
// boundary claim layers emptied
__global__ void k_slab_pack(const SlabArgs A)
{
    const uint32_t nij = (uint32_t)A.ni * (uint32_t)A.nj;
    const size_t nclaim = 4 * (size_t)nij;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < nclaim + 2 * (size_t)A.lw;
         q += (size_t)gridDim.x * blockDim.x) {
        if (q < nclaim) {
            const size_t layer = q / nij, w = q - layer * nij;
            const size_t L = layer < 2 ? layer : (size_t)A.m + layer - 2;   // 0, 1, m, m + 1
            A.claim[L * nij + w] = kNoClaim;
        } else {
            const size_t r = q - nclaim;
            const int side = r >= A.lw ? 1 : 0;
            const size_t w = r - (size_t)side * A.lw;
            const size_t L = side == 0 ? 1 : (size_t)A.m;
            uint32_t* bits = reinterpret_cast<uint32_t*>(A.send_commit[side] + slab_msg_bits_off(A.tcap));
            bits[w] = A.bits[L * A.lw + w];
        }
    }
}

// apply, step 1: the ghost layers take the neighbours' boundary bits
__global__ void k_slab_ghosts(const SlabArgs A)
{
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < 2 * (size_t)A.lw;
         q += (size_t)gridDim.x * blockDim.x) {
        const int side = q >= A.lw ? 1 : 0;
        if (!A.has[side]) continue;
        const size_t w = q - (size_t)side * A.lw;
        const size_t L = side == 0 ? 0 : (size_t)A.m + 1;
        A.bits[L * A.lw + w] = reinterpret_cast<const uint32_t*>(A.recv_commit[side] + slab_msg_bits_off(A.tcap))[w];
    }
}

// apply, step 2: the bits of this slab's own departures go back into the
// ghost layers (the neighbour sent its layer before placing them), the
// arrivals join the list and set their bits
__global__ void k_slab_arrivals(const SlabArgs A)
{
    const int nxt = A.cur ^ 1;
    const uint32_t nij = (uint32_t)A.ni * (uint32_t)A.nj;
    for (int side = 0; side < 2; ++side) {
        if (!A.has[side]) continue;
        const int nout = min(*reinterpret_cast<const int32_t*>(A.send_commit[side]), A.tcap);
        const SlabEntry* out = reinterpret_cast<const SlabEntry*>(A.send_commit[side] + slab_msg_entries_off());
        const int L_out = side == 0 ? 0 : A.m + 1;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nout; x += gridDim.x * blockDim.x)
            slab_set(A, out[x].i, out[x].j, L_out);
        const int nin = min(*reinterpret_cast<const int32_t*>(A.recv_commit[side]), A.tcap);
        const SlabEntry* in = reinterpret_cast<const SlabEntry*>(A.recv_commit[side] + slab_msg_entries_off());
        const int L_in = side == 0 ? 1 : A.m;
        for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nin; x += gridDim.x * blockDim.x) {
            const SlabEntry e = in[x];
            slab_set(A, e.i, e.j, L_in);
            const int o = atomicAdd(&A.count[nxt], 1);
            if (o < A.cap) {
                A.vox[nxt][o] = (int32_t)((uint32_t)e.i + (uint32_t)A.ni * (uint32_t)e.j + nij * (uint32_t)L_in);
                A.ids[nxt][o] = e.id;
                A.img[nxt][o] = e.img;
            } else {
                atomicOr(A.err, kErrListOverflow);
            }
        }
    }
}

// a new event's commit messages start empty; the buffer the next commit
// fills starts at zero molecules
__global__ void k_slab_begin(const SlabArgs A)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *reinterpret_cast<int32_t*>(A.send_commit[0]) = 0;
        *reinterpret_cast<int32_t*>(A.send_commit[1]) = 0;
        A.count[A.cur ^ 1] = 0;
    }
}

void launch_slab_claim(const SlabArgs& A, int blocks, cudaStream_t st)
{
    k_slab_begin<<<1, 32, 0, st>>>(A);
    k_slab_claim<<<blocks, 256, 0, st>>>(A);
}

void launch_slab_commit(const SlabArgs& A, int blocks, cudaStream_t st)
{
    k_slab_merge<<<blocks, 256, 0, st>>>(A);
    k_slab_commit<<<blocks, 256, 0, st>>>(A);
    k_slab_pack<<<blocks, 256, 0, st>>>(A);
}

void launch_slab_apply(const SlabArgs& A, int blocks, cudaStream_t st)
{
    k_slab_ghosts<<<blocks, 256, 0, st>>>(A);
    k_slab_arrivals<<<blocks, 256, 0, st>>>(A);
}
