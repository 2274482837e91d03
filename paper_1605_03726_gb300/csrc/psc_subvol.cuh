// psc_subvol.cuh -- the sub-volume rule (part of psc_kernels.cu's translation
// unit).  The paper's sub-volume scheme (Sec. 2.5) takes sub-volumes one after
// another in a random order so that those processed at the same time never
// touch each other.  On the lattice: sub-volumes of 2 x 2 x 2 voxels coloured
// by the parities of their indices (i/2, j/2, k/2); sub-volumes of one colour
// are at least one sub-volume apart, so a hop of one voxel from one of them
// never reaches what a hop from another reads or writes.  Per event: the eight
// colours in an order drawn for the event (Fisher-Yates, draw (a, g, s<<4 |
// kTagSubvol) for a = 7..1); within a colour, every sub-volume takes its
// molecules not yet processed in the event one at a time in ascending id,
// each seeing the grid as left before it.
//
// A molecule moves only when its colour's turn comes, so the sub-volume it is
// processed in is the one it stands in when the event begins.  Each event:
//   pass 0   every molecule notes its colour and sub-volume; one alone in its
//            sub-volume (one of the sub-volume's 8 bits set: at the start of
//            the event only waiting molecules stand there) leads it by
//            itself, the others offer their id to the sub-volume's word
//            (atomicMin) and join the sub-volume's chain (a linked list
//            through the list slots);
//   pass 1   the lowest id of each sub-volume (its leader) enters the list of
//            leaders of its colour (one counter per colour and block);
//   turns    for each colour in the drawn order, every leader of the colour
//            walks its chain (at most 8 molecules), sorts it by id and hops
//            the molecules one after another (Sec. 2.3) against the current
//            grid, then frees the word and the chain.
// Bounded grid barriers separate the passes and the turns (10 per event).
// A leader moves molecules of other list slots, so everything the list holds
// is read past L1.  Species without reactions only.

constexpr uint32_t kTagSubvol = 3u;

// the 8 bits of the 2x2x2 sub-volume holding voxel (i, j, k) in its mirror
// word (bricks are 4 x 4 x 2 voxels, so a sub-volume never straddles two)
__device__ __forceinline__ uint32_t subvol_mask(int32_t i, int32_t j, int32_t k)
{
    const uint32_t bx = (uint32_t)i & 2u, by = ((uint32_t)j & 2u) << 2;   // bit offsets of the 2 x 2 corner
    const uint32_t row = 3u << bx;                                          // two voxels along i
    const uint32_t layer = (row | (row << 4)) << by;                        // two rows along j
    (void)k;
    return layer | (layer << 16);                                           // both k layers of the brick
}

__device__ __forceinline__ int subvol_colour(int32_t i, int32_t j, int32_t k)
{
    return ((i >> 1) & 1) | (((j >> 1) & 1) << 1) | (((k >> 1) & 1) << 2);
}

// one hop of the molecule in list slot x at (i, j, k) (bit bp) against the
// current grid; returns 1 if it moved
__device__ __forceinline__ int subvol_hop(const EventArgs& a, const Geometry& G, int x, uint32_t id, uint32_t g,
                                          uint32_t c2, int32_t i, int32_t j, int32_t k, BitPos bp)
{
    uint32_t u[4];
    philox(id, g, c2, 0u, a.key0, a.key1, u);
    const int d = (int)__umulhi(u[0], 12u);
    Nb nb;
    if (!neighbor(G, i, j, k, d, nb)) return 0;                       // wall
    const BitPos bt = bitpos(G, nb.i, nb.j, nb.k);
    if (__ldcg(&a.bits[bt.word]) & bt.mask) return 0;                  // occupied
    bit_move(a.bits, bp, bt);
    a.list.vox[x] = nb.t;
    if (nb.wrap) a.list.img[x] = img_add(__ldcg((const unsigned long long*)&a.list.img[x]), nb.wrap);
    return 1;
}

constexpr uint32_t kSubvolLeader = 0x80000000u;     // state bit: the slot leads its sub-volume
constexpr uint32_t kSubvolAlone = 0x40000000u;      // state bit: ... and is alone in it (no chain)

__global__ void __launch_bounds__(256) k_subvol_run(const SubvolArgs A)
{
    const EventArgs& a = A.ev;
    const Geometry& G = a.geo;
    __shared__ int s_order[8];
    __shared__ uint32_t s_cnt[8], s_base[8], s_off[9];
    const int n = *a.count;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, T = gridDim.x * blockDim.x;
    const uint32_t c2 = ((uint32_t)a.s << 4) | kTagEvent;
    const uint32_t sub_nbi = (uint32_t)((G.ni + 1) / 2), sub_nbj = (uint32_t)((G.nj + 1) / 2);
    unsigned long long n_hop = 0;
    for (int e = 0; e < A.n_events; ++e) {
        const uint32_t g = a.g + (uint32_t)e;
        uint32_t* cnt = A.counters + (e & 1) * 16;       // [0, 8) molecules, [8, 16) leaders per colour
        if (threadIdx.x == 0) {
            int ord[8] = {0, 1, 2, 3, 4, 5, 6, 7};
            for (int q = 7; q > 0; --q) {
                uint32_t u[4];
                philox((uint32_t)q, g, ((uint32_t)a.s << 4) | kTagSubvol, 0u, a.key0, a.key1, u);
                const int r = (int)__umulhi(u[0], (uint32_t)(q + 1));
                const int t = ord[q]; ord[q] = ord[r]; ord[r] = t;
            }
            for (int q = 0; q < 8; ++q) s_order[q] = ord[q];
        }
        if (threadIdx.x < 8) s_cnt[threadIdx.x] = 0u;
        __syncthreads();
        // pass 0: colour, sub-volume, offer and chain
        for (int x = gt; x < n; x += T) {
            int32_t i, j, k;
            decode(G, (uint32_t)__ldcg(&a.list.vox[x]), i, j, k);
            const int c = subvol_colour(i, j, k);
            const uint32_t sv = ((uint32_t)(k >> 1) * sub_nbj + (uint32_t)(j >> 1)) * sub_nbi + (uint32_t)(i >> 1);
            A.colour0[x] = (uint8_t)c;
            const BitPos bp = bitpos(G, i, j, k);
            if (__popc(__ldcg(&a.bits[bp.word]) & subvol_mask(i, j, k)) == 1) {
                A.state[x] = sv | kSubvolLeader | kSubvolAlone;
            } else {
                A.state[x] = sv;
                atomicMin(&A.word[sv], a.list.ids[x]);
                A.next[x] = atomicExch(&A.head[sv], (uint32_t)x);
            }
            atomicAdd(&s_cnt[c], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 8 && s_cnt[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], s_cnt[threadIdx.x]);
        if (!grid_barrier(A.barrier, &a.sc->err, A.barrier_timeout_ns, A.barrier_phantom)) return;
        if (gt < 16) A.counters[((e + 1) & 1) * 16 + gt] = 0u;   // for the next event
        if (threadIdx.x == 0) {
            uint32_t o = 0;
            for (int c = 0; c < 8; ++c) { s_off[c] = o; o += __ldcg(&cnt[c]); }
            s_off[8] = o;
        }
        if (threadIdx.x < 8) s_cnt[threadIdx.x] = 0u;
        __syncthreads();
        // pass 1: leaders into their colour's list (a block's share reserved at once)
        for (int x = gt; x < n; x += T) {
            const uint32_t st = A.state[x];
            if (!(st & kSubvolLeader)) {
                if (__ldcg(&A.word[st]) != a.list.ids[x]) continue;
                A.state[x] = st | kSubvolLeader;
            }
            atomicAdd(&s_cnt[A.colour0[x]], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 8) {
            s_base[threadIdx.x] = s_cnt[threadIdx.x] ? atomicAdd(&cnt[8 + threadIdx.x], s_cnt[threadIdx.x]) : 0u;
            s_cnt[threadIdx.x] = 0u;
        }
        __syncthreads();
        for (int x = gt; x < n; x += T) {
            const uint32_t st = A.state[x];
            if (!(st & kSubvolLeader)) continue;
            const int c = A.colour0[x];
            const uint32_t at = s_off[c] + s_base[c] + atomicAdd(&s_cnt[c], 1u);
            // the slot (top bit: alone) and, for one alone, its voxel, read together in its turn
            A.lead[at] = (uint32_t)x | (st & kSubvolAlone ? kSubvolLeader : 0u);
            if (st & kSubvolAlone) A.lead_vox[at] = (uint32_t)__ldcg(&a.list.vox[x]);
        }
        if (!grid_barrier(A.barrier, &a.sc->err, A.barrier_timeout_ns, A.barrier_phantom)) return;
        // the colours' turns
        for (int ci = 0; ci < 8; ++ci) {
            const int c = s_order[ci];
            const uint32_t nl = __ldcg(&cnt[8 + c]), base = s_off[c];
            for (uint32_t q = (uint32_t)gt; q < nl; q += (uint32_t)T) {
                const uint32_t lx = __ldcg(&A.lead[base + q]);
                if (lx & kSubvolLeader) {                         // alone: no chain
                    const uint32_t x = lx & ~kSubvolLeader;
                    int32_t i, j, k;
                    decode(G, __ldcg(&A.lead_vox[base + q]), i, j, k);
                    n_hop += (unsigned long long)subvol_hop(a, G, (int)x, a.list.ids[x], g, c2, i, j, k,
                                                            bitpos(G, i, j, k));
                    continue;
                }
                const uint32_t sv = __ldcg(&A.state[lx]) & ~kSubvolLeader;
                uint32_t ids[8], slots[8];
                int m = 0;
                for (uint32_t p = __ldcg(&A.head[sv]); p != kNoClaim; p = __ldcg(&A.next[p])) {
                    if (m == 8 || p >= (uint32_t)n) {             // a sub-volume holds at most 8
                        atomicOr(&a.sc->err, kErrListOverflow);
                        break;
                    }
                    ids[m] = a.list.ids[p];
                    slots[m] = p;
                    ++m;
                }
                for (int r0 = 1; r0 < m; ++r0) {                  // ascending id
                    const uint32_t ki = ids[r0], ks = slots[r0];
                    int r = r0 - 1;
                    while (r >= 0 && ids[r] > ki) { ids[r + 1] = ids[r]; slots[r + 1] = slots[r]; --r; }
                    ids[r + 1] = ki;
                    slots[r + 1] = ks;
                }
                for (int r = 0; r < m; ++r) {
                    int32_t i, j, k;
                    decode(G, (uint32_t)__ldcg(&a.list.vox[slots[r]]), i, j, k);
                    n_hop += (unsigned long long)subvol_hop(a, G, (int)slots[r], ids[r], g, c2, i, j, k,
                                                            bitpos(G, i, j, k));
                }
                A.head[sv] = kNoClaim;
                A.word[sv] = kNoClaim;
            }
            if (!grid_barrier(A.barrier, &a.sc->err, A.barrier_timeout_ns, A.barrier_phantom)) return;
        }
    }
    if (a.collect_stats) {
        flush_stat(&a.sc->stats[kStatHops], n_hop);
        if (gt == 0) atomicAdd(&a.sc->stats[kStatAttempts], (unsigned long long)n * (unsigned long long)A.n_events);
    }
}

cudaError_t launch_subvol(const SubvolArgs& A, int blocks, int threads, cudaStream_t st)
{
    void* args[] = {const_cast<SubvolArgs*>(&A)};
    return cudaLaunchCooperativeKernel((const void*)k_subvol_run, dim3(blocks), dim3(threads), args, 0, st);
}

int subvol_max_blocks(int sm_count)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_subvol_run, 256, 0) != cudaSuccess) return 0;
    return (nb < 4 ? nb : 4) * sm_count;
}
