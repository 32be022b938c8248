// Tile bucketing and per-tile depth sort of (Gaussian, tile) pairs and of query points.
//
// k_bin_append (preprocess.cu) leaves an unsorted list of (tile, depth key, record) and a count
// per tile. Here: the counts are scanned into per-tile ranges, k_bucket scatters each pair into
// its tile's range as one 64-bit word (depth key bits << 32 | record), and k_tile_sort sorts each
// tile's range ascending with one CTA per tile. The depth keys are non-negative floats, so their
// bits order like their values; the record index in the low word breaks ties deterministically.
//
// k_tile_sort is a bitonic network in its ascending-only form (the first exchange of every merge
// compares i with i ^ (k - 1), all later ones i with i ^ j, and every exchange keeps the smaller
// word at the lower index). With that form, positions past the end behave as +infinity and are
// never exchanged, so any length works without padding in memory. Up to kSortCap words are sorted
// in shared memory at once; longer ranges run the exchanges with j >= kSortCap in global memory
// and finish each kSortCap-aligned block in shared memory.
#include "sof_internal.cuh"

namespace sof {
namespace {

// Two configurations: ranges of up to 4096 words in a 256-thread CTA with 32 KB of shared memory
// (many CTAs per SM), longer ones in a 512-thread CTA with 64 KB blocks.
constexpr int kSmallCap = 4096, kSmallThreads = 256;
constexpr int kLargeCap = 8192, kLargeThreads = 512;

__global__ void k_ranges_from_counts(const int *__restrict__ counts, const int *__restrict__ offsets, int n_tiles,
                                     int2 *__restrict__ ranges, int *__restrict__ cursor) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    const int o = offsets[t];
    ranges[t] = make_int2(o, o + counts[t]);
    cursor[t] = o;
}

__global__ void k_bucket(const unsigned *__restrict__ ptile, const unsigned *__restrict__ pkey,
                         const unsigned *__restrict__ prec, const int *__restrict__ n_dev, long long cap,
                         int *__restrict__ cursor, unsigned long long *__restrict__ pairs,
                         unsigned long long *__restrict__ pair_total) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = min((long long)*n_dev, cap);
    if (i == 0 && pair_total) atomicAdd(pair_total, (unsigned long long)n);
    if (i >= n) return;
    const int pos = atomicAdd(&cursor[ptile[i]], 1);
    pairs[pos] = ((unsigned long long)pkey[i] << 32) | (unsigned long long)prec[i];
}

// One compare-exchange of the ascending network: lower element lo, partner hi > lo.
__device__ __forceinline__ void cx(unsigned long long *a, int lo, int hi) {
    const unsigned long long x = a[lo], y = a[hi];
    if (y < x) {
        a[lo] = y;
        a[hi] = x;
    }
}

// Lower element of the i-th exchange at distance j (insert a zero bit at position log2 j).
__device__ __forceinline__ int lower_of(int i, int j) { return ((i & ~(j - 1)) << 1) | (i & (j - 1)); }

// Exchanges of one step (k, j) over positions [0, n) of a (in shared or global memory); the first
// step of each merge (j == k / 2) mirrors across the k-block.
template <int THREADS>
__device__ __forceinline__ void bitonic_step(unsigned long long *a, int n, int P, int k, int j) {
    for (int i = threadIdx.x; i < P / 2; i += THREADS) {
        const int lo = lower_of(i, j);
        const int hi = (j == (k >> 1)) ? (lo ^ (k - 1)) : (lo + j);
        if (hi < n) cx(a, lo, hi);
    }
}

// Steps j = jstart, jstart / 2, ..., 1 of merge k on the shared-memory copy of one block.
template <int THREADS>
__device__ void smem_steps(unsigned long long *s, int nb, int Pb, int k, int jstart) {
    for (int j = jstart; j > 0; j >>= 1) {
        bitonic_step<THREADS>(s, nb, Pb, k, j);
        __syncthreads();
    }
}

// Sorts the ranges of length in (lo_len, hi_len]; the others are left to the other configuration.
template <int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS) k_tile_sort(const int2 *__restrict__ ranges,
                                                       unsigned long long *__restrict__ pairs, int lo_len, int hi_len) {
    extern __shared__ unsigned long long s[];  // [CAP]
    const int2 rg = ranges[blockIdx.x];
    const int n = rg.y - rg.x;
    if (n <= 1 || n <= lo_len || n > hi_len) return;
    unsigned long long *a = pairs + rg.x;
    int P = 1;
    while (P < n) P <<= 1;
    // 1. every CAP block sorted on its own, in shared memory
    const int B = P < CAP ? P : CAP;
    for (int b0 = 0; b0 < n; b0 += B) {
        const int nb = min(B, n - b0);
        for (int i = threadIdx.x; i < nb; i += THREADS) s[i] = a[b0 + i];
        __syncthreads();
        for (int k = 2; k <= B; k <<= 1) smem_steps<THREADS>(s, nb, B, k, k >> 1);
        for (int i = threadIdx.x; i < nb; i += THREADS) a[b0 + i] = s[i];
        __syncthreads();
    }
    // 2. merges longer than a block: the exchanges at distance >= CAP in global memory, the rest
    //    per block in shared memory
    for (int k = 2 * B; k <= P; k <<= 1) {
        int j = k >> 1;
        for (; j >= B; j >>= 1) {
            bitonic_step<THREADS>(a, n, P, k, j);
            __syncthreads();
        }
        for (int b0 = 0; b0 < n; b0 += B) {
            const int nb = min(B, n - b0);
            for (int i = threadIdx.x; i < nb; i += THREADS) s[i] = a[b0 + i];
            __syncthreads();
            smem_steps<THREADS>(s, nb, B, 2 * B, j);  // plain (non-mirrored) steps j < B
            for (int i = threadIdx.x; i < nb; i += THREADS) a[b0 + i] = s[i];
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t launch_tile_buckets(const unsigned *ptile, const unsigned *pkey, const unsigned *prec,
                                const int *n_dev, long long cap, const int *tile_counts,
                                const int *tile_offsets, int n_tiles, int2 *ranges, int *cursor,
                                unsigned long long *pairs, unsigned long long *pair_total, cudaStream_t s) {
    if (n_tiles <= 0) return cudaSuccess;
    note_launches(3);
    k_ranges_from_counts<<<(n_tiles + 255) / 256, 256, 0, s>>>(tile_counts, tile_offsets, n_tiles, ranges, cursor);
    if (cap > 0)
        k_bucket<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(ptile, pkey, prec, n_dev, cap, cursor, pairs,
                                                               pair_total);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_sort<kLargeCap, kLargeThreads>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(kLargeCap * sizeof(unsigned long long)));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    note_launches(1);
    k_tile_sort<kSmallCap, kSmallThreads><<<n_tiles, kSmallThreads, kSmallCap * sizeof(unsigned long long), s>>>(
        ranges, pairs, 0, kSmallCap);
    k_tile_sort<kLargeCap, kLargeThreads><<<n_tiles, kLargeThreads, kLargeCap * sizeof(unsigned long long), s>>>(
        ranges, pairs, kSmallCap, 1 << 30);
    return cudaGetLastError();
}

}  // namespace sof
