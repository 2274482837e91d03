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
// each seeing the grid as left before it.  All sub-volumes of a colour work at
// once, one molecule each per round:
//   round, phase A   each waiting molecule of the colour counts itself; if its
//                    sub-volume holds other molecules it offers its id to the
//                    sub-volume's word (atomicMin; alone it is the lowest);
//   phase B          the lowest waiting id of each sub-volume hops (Sec. 2.3)
//                    against the current grid and is done for the event;
// until a round finds nobody waiting.  Grid barriers (bounded) separate the
// phases.  Species without reactions only.

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

__global__ void __launch_bounds__(256) k_subvol_run(const SubvolArgs A)
{
    const EventArgs& a = A.ev;
    const Geometry& G = a.geo;
    __shared__ int s_order[8];
    const int n = *a.count;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x, T = gridDim.x * blockDim.x;
    const uint32_t c2 = ((uint32_t)a.s << 4) | kTagEvent;
    const uint32_t sub_nbi = (uint32_t)((G.ni + 1) / 2), sub_nbj = (uint32_t)((G.nj + 1) / 2);
    unsigned long long n_hop = 0;
    uint32_t k_round = 0;                                // rounds so far in the launch (rotates the counters)
    for (int e = 0; e < A.n_events; ++e) {
        const uint32_t g = a.g + (uint32_t)e;
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
        __syncthreads();
        for (int ci = 0; ci < 8; ++ci) {
            const int colour = s_order[ci];
            for (uint32_t r = 0;; ++r) {
                uint32_t* word = A.word[r & 1u];
                uint32_t* prev = A.word[(r & 1u) ^ 1u];
                uint32_t* cnt = &A.count[k_round % 3u];
                if (gt == 0) A.count[(k_round + 1u) % 3u] = 0u;
                // phase A: count the waiting molecules of the colour; in a
                // sub-volume holding several, offer the id to its word
                unsigned int waiting = 0;
                for (int x = gt; x < n; x += T) {
                    const uint32_t w = A.won[x];
                    if (w) {                              // won last round: its word is free again
                        prev[w - 1u] = kNoClaim;
                        A.won[x] = 0u;
                    }
                    if (A.done[x] == g + 1u) continue;
                    int32_t i, j, k;
                    decode(G, (uint32_t)a.list.vox[x], i, j, k);
                    if (subvol_colour(i, j, k) != colour) continue;
                    ++waiting;
                    const BitPos bp = bitpos(G, i, j, k);
                    const bool alone = __popc(__ldcg(&a.bits[bp.word]) & subvol_mask(i, j, k)) == 1;
                    A.alone[x] = alone ? 1u : 0u;
                    if (!alone) {
                        const uint32_t sv = ((uint32_t)(k >> 1) * sub_nbj + (uint32_t)(j >> 1)) * sub_nbi + (uint32_t)(i >> 1);
                        atomicMin(&word[sv], a.list.ids[x]);
                    }
                }
                waiting = __reduce_add_sync(0xFFFFFFFFu, waiting);
                if ((threadIdx.x & 31) == 0 && waiting) atomicAdd(cnt, waiting);
                ++k_round;
                if (!grid_barrier(A.barrier, &a.sc->err, A.barrier_timeout_ns, A.barrier_phantom)) return;
                if (*((volatile uint32_t*)cnt) == 0u) break;          // the colour is finished
                // phase B: the lowest waiting id of every sub-volume hops
                for (int x = gt; x < n; x += T) {
                    if (A.done[x] == g + 1u) continue;
                    int32_t i, j, k;
                    const uint32_t v = (uint32_t)a.list.vox[x];
                    decode(G, v, i, j, k);
                    if (subvol_colour(i, j, k) != colour) continue;
                    const uint32_t id = a.list.ids[x];
                    const uint32_t sv = ((uint32_t)(k >> 1) * sub_nbj + (uint32_t)(j >> 1)) * sub_nbi + (uint32_t)(i >> 1);
                    const bool alone = A.alone[x] != 0u;
                    if (!alone && __ldcg(&word[sv]) != id) continue;   // a lower id of the sub-volume goes first
                    A.done[x] = g + 1u;
                    if (!alone) A.won[x] = sv + 1u;       // its word is reset next round
                    uint32_t u[4];
                    philox(id, g, c2, 0u, a.key0, a.key1, u);
                    const int d = (int)__umulhi(u[0], 12u);
                    Nb nb;
                    if (!neighbor(G, i, j, k, d, nb)) continue;                 // wall
                    const BitPos bp = bitpos(G, i, j, k), bt = bitpos(G, nb.i, nb.j, nb.k);
                    if (__ldcg(&a.bits[bt.word]) & bt.mask) continue;           // occupied
                    bit_move(a.bits, bp, bt);
                    a.list.vox[x] = nb.t;
                    if (nb.wrap) a.list.img[x] = img_add(a.list.img[x], nb.wrap);
                    ++n_hop;
                }
                if (!grid_barrier(A.barrier, &a.sc->err, A.barrier_timeout_ns, A.barrier_phantom)) return;
            }
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
