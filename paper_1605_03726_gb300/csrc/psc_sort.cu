// psc_sort.cu -- stable LSD radix sort of (uint32 key, uint32 value) pairs.
//
// Used for the placement of molecules (voxels ordered by their Philox key; a
// stable sort of keys in voxel order gives the (key, voxel) order) and for the
// periodic Morton re-sort of the molecule lists.  Each 8-bit pass is
//   hist     per-tile digit counts, stored digit-major;
//   scan     exclusive scan of the counts (three kernels);
//   scatter  per tile, stable ranks from warp match + per-warp prefix counts.
// The element count may live on the device so that no host sync is needed.
#include "psc_internal.h"

namespace psc {

constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;   // 4096 keys per tile
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;    // 4096 counts per scan tile

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t sort_scratch_bytes(int64_t max_n)
{
    const int64_t tiles = ceil_div(max_n > 0 ? max_n : 1, kSortTile);
    const int64_t hist = 256 * tiles;
    const int64_t sums = ceil_div(hist, kScanTile);
    return 2 * align256((size_t)max_n * 4) + align256((size_t)hist * 4) + align256((size_t)sums * 4);
}

void sort_scratch_bind(SortScratch& s, void* base, int64_t max_n)
{
    char* p = static_cast<char*>(base);
    const int64_t tiles = ceil_div(max_n > 0 ? max_n : 1, kSortTile);
    s.max_n = max_n;
    s.hist_len = 256 * tiles;
    s.sums_len = ceil_div(s.hist_len, kScanTile);
    s.keys_alt = reinterpret_cast<uint32_t*>(p); p += align256((size_t)max_n * 4);
    s.vals_alt = reinterpret_cast<uint32_t*>(p); p += align256((size_t)max_n * 4);
    s.hist = reinterpret_cast<uint32_t*>(p); p += align256((size_t)s.hist_len * 4);
    s.block_sums = reinterpret_cast<uint32_t*>(p);
}

// the element count: n_host, or the count in device memory capped at n_host
__device__ __forceinline__ int64_t sort_n(const int32_t* n_dev, int64_t n_host)
{
    return n_dev ? min((int64_t)*n_dev, n_host) : n_host;
}

__global__ void __launch_bounds__(kSortThreads)
k_hist(const uint32_t* keys, const int32_t* n_dev, int64_t n_host, int shift, uint32_t* hist, int tiles)
{
    __shared__ uint32_t h[256];
    const int64_t n = sort_n(n_dev, n_host);
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t start = (int64_t)blockIdx.x * kSortTile;
    const int64_t end = start + kSortTile < n ? start + kSortTile : n;
    for (int64_t x = start + threadIdx.x; x < end; x += kSortThreads)
        atomicAdd(&h[(keys[x] >> shift) & 255u], 1u);
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// ---- exclusive scan of hist (length len) ----
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot, uint32_t& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t w = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) warp_tot[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    total = warp_tot[(blockDim.x >> 5) - 1];
    const uint32_t before = warp ? warp_tot[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* in, int64_t len, uint32_t* sums)
{
    __shared__ uint32_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < len) s += in[base + q];
    uint32_t total;
    block_exclusive_scan(s, wt, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// single block: exclusive scan of sums in place (len <= many thousands)
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t* sums, int64_t len)
{
    __shared__ uint32_t wt[32];
    uint32_t carry = 0;
    for (int64_t base = 0; base < len; base += kScanThreads) {
        const int64_t x = base + threadIdx.x;
        const uint32_t v = x < len ? sums[x] : 0;
        uint32_t total;
        const uint32_t e = block_exclusive_scan(v, wt, total);
        if (x < len) sums[x] = carry + e;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_down(uint32_t* data, int64_t len, const uint32_t* sums)
{
    __shared__ uint32_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        v[q] = base + q < len ? data[base + q] : 0;
        s += v[q];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, wt, total) + sums[blockIdx.x];
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q < len) data[base + q] = run;
        run += v[q];
    }
}

// ---- stable scatter ----
__global__ void __launch_bounds__(kSortThreads)
k_scatter(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
          const int32_t* n_dev, int64_t n_host, int shift, const uint32_t* offsets, int tiles)
{
    __shared__ uint32_t base[256];
    __shared__ uint32_t running[256];
    __shared__ uint32_t wcount[kSortThreads / 32][256];
    const int64_t n = sort_n(n_dev, n_host);
    const int64_t start = (int64_t)blockIdx.x * kSortTile;
    if (start >= n) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offsets[(int64_t)tid * tiles + blockIdx.x];
    running[tid] = 0;
    const unsigned lt = (1u << lane) - 1u;
    for (int round = 0; round < kSortRounds; ++round) {
        const int64_t x = start + (int64_t)round * kSortThreads + tid;
        const bool valid = x < n;
        const uint32_t key = valid ? keys_in[x] : 0u;
        const uint32_t val = valid ? vals_in[x] : 0u;
        const uint32_t d = (key >> shift) & 255u;
        for (int q = tid; q < (kSortThreads / 32) * 256; q += kSortThreads) (&wcount[0][0])[q] = 0;
        __syncthreads();
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, valid ? d : 256u);
        const uint32_t rank = __popc(peers & lt);
        if (valid && lane == __ffs(peers) - 1) wcount[warp][d] = __popc(peers);
        __syncthreads();
        {   // thread tid owns digit tid: prefix over warps, carried over rounds
            uint32_t acc = running[tid];
#pragma unroll
            for (int w = 0; w < kSortThreads / 32; ++w) {
                const uint32_t c = wcount[w][tid];
                wcount[w][tid] = acc;
                acc += c;
            }
            running[tid] = acc;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = base[d] + wcount[warp][d] + rank;
            keys_out[pos] = key;
            vals_out[pos] = val;
        }
        __syncthreads();
    }
}

int radix_sort_pairs(uint32_t* keys, uint32_t* vals, const int32_t* n_dev, int64_t n_host,
                     int64_t max_n, int bits, SortScratch& s, cudaStream_t st, int64_t* launches)
{
    if (max_n <= 0) return 0;
    if (max_n > s.max_n) return -1;
    const int tiles = (int)ceil_div(max_n, kSortTile);
    const int64_t hist_len = 256 * (int64_t)tiles;
    const int scan_blocks = (int)ceil_div(hist_len, kScanTile);
    int passes = (bits + 7) / 8;
    if (passes & 1) ++passes;           // even: the result lands back in (keys, vals)
    uint32_t *ki = keys, *vi = vals, *ko = s.keys_alt, *vo = s.vals_alt;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_hist<<<tiles, kSortThreads, 0, st>>>(ki, n_dev, n_host, shift, s.hist, tiles);
        k_scan_reduce<<<scan_blocks, kScanThreads, 0, st>>>(s.hist, hist_len, s.block_sums);
        k_scan_sums<<<1, kScanThreads, 0, st>>>(s.block_sums, scan_blocks);
        k_scan_down<<<scan_blocks, kScanThreads, 0, st>>>(s.hist, hist_len, s.block_sums);
        k_scatter<<<tiles, kSortThreads, 0, st>>>(ki, vi, ko, vo, n_dev, n_host, shift, s.hist, tiles);
        if (launches) *launches += 5;
        uint32_t* t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    return cudaPeekAtLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace psc
