// psc_readout.cu -- the molecules of one list in id order, built on the
// device for the read-out calls (psc_coords, psc_unwrapped): the list's ids
// are sorted together with their list slots (the radix sort of psc_sort.cu),
// then one gather writes every molecule's coordinates and id, in id order,
// into a staging buffer that the host copies in one piece.
#include "psc_readout.h"

namespace psc {

__global__ void k_id_keys(const uint32_t* ids, int32_t n, uint32_t* keys, uint32_t* slots)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        keys[r] = ids[r];
        slots[r] = (uint32_t)r;
    }
}

// entry a of the output is list slot perm[a]: (i, j, k) from its voxel index
// v = i + ni (j + nj k), or, unwrapped, the integer basis (X, Y, Z) of its
// lattice point with the wrap counters of its periodic crossings (psc.h)
__global__ void k_gather_positions(const SpeciesList list, const uint32_t* perm, int32_t n, int32_t ni, int32_t nj,
                                   int32_t nk, int unwrapped, int fcc, int32_t* out, uint32_t* out_ids)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        const uint32_t p = perm[a];
        const uint32_t v = (uint32_t)list.vox[p], q = v / (uint32_t)ni;
        const int32_t i = (int32_t)(v - q * (uint32_t)ni), j = (int32_t)(q % (uint32_t)nj),
                      k = (int32_t)(q / (uint32_t)nj);
        if (!unwrapped) {
            out[3 * a + 0] = i;
            out[3 * a + 1] = j;
            out[3 * a + 2] = k;
        } else {
            const uint64_t w = list.img[p];
            const int32_t I = i + (int32_t)(int16_t)(w & 0xFFFF) * ni;
            const int32_t J = j + (int32_t)(int16_t)((w >> 16) & 0xFFFF) * nj;
            const int32_t K = k + (int32_t)(int16_t)((w >> 32) & 0xFFFF) * nk;
            if (fcc) {
                const int32_t c3 = ((K % 3) + 3) % 3;
                out[3 * a + 0] = 2 * I + ((J + (c3 == 1 ? 1 : 0)) & 1);
                out[3 * a + 1] = 3 * J + c3;
            } else {
                out[3 * a + 0] = 2 * I + ((J + K) & 1);
                out[3 * a + 1] = 3 * J + (K & 1);
            }
            out[3 * a + 2] = K;
        }
        out_ids[a] = list.ids[p];
    }
}

int readout_positions(const SpeciesList& list, int32_t n, int32_t ni, int32_t nj, int32_t nk, bool unwrapped,
                      bool fcc, uint32_t* keys, uint32_t* slots, SortScratch& scratch, int32_t* out,
                      uint32_t* out_ids, int blocks, cudaStream_t st, int64_t* launches)
{
    if (n <= 0) return 0;
    k_id_keys<<<blocks, 256, 0, st>>>(list.ids, n, keys, slots);
    if (radix_sort_pairs(keys, slots, nullptr, n, n, 32, scratch, st, launches) != 0) return -1;
    k_gather_positions<<<blocks, 256, 0, st>>>(list, slots, n, ni, nj, nk, unwrapped ? 1 : 0, fcc ? 1 : 0, out,
                                               out_ids);
    if (launches) *launches += 2;
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace psc
