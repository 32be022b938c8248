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
//
// Render calls sort only the front of each tile's list up front (k_tile_select): a pixel stops once
// its transmittance falls below t_stop, after a few hundred of its tile's records at most, so most
// of a long list is never read. The front is every word whose key lies at or below a threshold
// chosen by a two-level histogram of the key bits (at least `prefix` words); it is sorted and
// followed by the rest of the list unsorted. The composite's first pass reads the front only and
// merges against the threshold as the key that follows it. Pixels still open at the threshold are
// redone by the second pass, after k_tile_sort has sorted the rest of their tiles' lists (every key
// there is above every key of the front, so the whole list is then in order).
#include <math.h>

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
                         const unsigned *__restrict__ prec, const unsigned long long *__restrict__ n_dev, long long cap,
                         int *__restrict__ cursor, unsigned long long *__restrict__ pairs,
                         unsigned long long *__restrict__ pair_total, const unsigned *__restrict__ prank,
                         const int *__restrict__ tile_offsets) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)min(*n_dev, (unsigned long long)cap);
    if (i == 0 && pair_total) atomicAdd(pair_total, (unsigned long long)n);
    if (i >= n) return;
    const unsigned t = ptile[i];
    // with the ranks the append took, each pair has its place: no atomic per pair
    const int pos = prank ? tile_offsets[t] + (int)prank[i] : atomicAdd(&cursor[t], 1);
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

// Bitonic sort of s[0, n) in shared memory (n <= THREADS * anything; P the power of two >= n).
template <int THREADS>
__device__ void smem_sort(unsigned long long *s, int n) {
    int P = 1;
    while (P < n) P <<= 1;
    for (int k = 2; k <= P; k <<= 1) smem_steps<THREADS>(s, n, P, k, k >> 1);
}

// Sorts a[0, n) (any n) with one CTA: CAP-word blocks in shared memory s[CAP], the exchanges at
// distance >= CAP of longer merges in global memory.
// With blocks_only, only step 1 runs: every CAP-word block is sorted, the blocks are not merged.
template <int CAP, int THREADS>
__device__ void sort_range(unsigned long long *a, int n, unsigned long long *s, bool blocks_only = false) {
    if (n <= 1) return;
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
    if (blocks_only) return;
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

// Stable LSD radix sort of s[0, n) (n <= CAP) by the key (high word), 8-bit digits, followed by the
// ordering of every run of equal keys by record (low word): the result is the ascending order of the
// whole 64-bit words, whatever order the bucketing's atomics left them in.
// Each pass keeps the words in registers, warp-striped: warp w holds positions [w seg, (w+1) seg)
// (seg = n / warps rounded up to 32, so short ranges still spread over every warp), lane l of it
// positions w seg + 32 j + l. The warp ranks one 32-word step at a time
// (lanes with equal digits found by eight ballots), so the scatter back into s is stable. A pass
// whose digit is the same for every word is skipped.
template <int CAP, int THREADS>
struct RadixSmem {
    static constexpr int W = THREADS / 32, ITEMS = CAP / THREADS, SEG = ITEMS * 32;
    unsigned long long s[CAP];
    unsigned cnt[W][256];  // per warp and digit: count, then the warp's next scatter position
    unsigned tot[256];
    int wsum[8];
    int skip[4];            // per pass: one digit holds every word
    int runs[64];           // starts of runs of equal keys longer than kRunSerial
    int n_runs;
};

constexpr int kRunSerial = 32;  // runs of equal keys up to this length are ordered by one thread

template <int CAP, int THREADS>
__device__ void smem_radix_sort(RadixSmem<CAP, THREADS> &S, int n, bool coarse) {
    using RS = RadixSmem<CAP, THREADS>;
    constexpr int W = RS::W, ITEMS = RS::ITEMS;
    static_assert(THREADS >= 256 && THREADS % 256 == 0, "one thread per digit in the scan");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int seg = ((n + W - 1) / W + 31) & ~31;  // <= SEG for n <= CAP
    const int s0 = warp * seg, s1 = min(n, s0 + seg);
    if (tid < 4) S.skip[tid] = 0;
    __syncthreads();
    for (int pass = coarse ? 2 : 0; pass < 4; ++pass) {
        const int shift = 32 + 8 * pass;
        unsigned long long w[ITEMS];
        unsigned peers[ITEMS];
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const int i = s0 + j * 32 + lane;
            w[j] = i < s1 ? S.s[i] : ~0ull;
        }
        for (int d = lane; d < 256; d += 32) S.cnt[warp][d] = 0u;
        __syncwarp();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            peers[j] = 0u;
            if (s0 + j * 32 >= s1) continue;  // uniform over the warp
            const bool valid = s0 + j * 32 + lane < s1;
            const unsigned d = (unsigned)(w[j] >> shift) & 255u;
            unsigned m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                m &= ((d >> b) & 1u) ? bb : ~bb;
            }
            peers[j] = m;
            if (valid && (m & lt) == 0u) S.cnt[warp][d] += (unsigned)__popc(m);
            __syncwarp();
        }
        __syncthreads();
        // exclusive offsets, digit-major and warp-minor: stable across warps
        if (tid < 256) {
            unsigned run = 0;
#pragma unroll
            for (int u = 0; u < W; ++u) {
                const unsigned c = S.cnt[u][tid];
                S.cnt[u][tid] = run;
                run += c;
            }
            S.tot[tid] = run;
            if (run == (unsigned)n) S.skip[pass] = 1;  // one digit holds every word: nothing moves
            unsigned inc = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) S.wsum[warp] = (int)inc;
            S.tot[tid] = inc - run;  // exclusive within the warp's 32 digits
        }
        __syncthreads();
        if (S.skip[pass]) continue;  // uniform: the words stay where they are
        if (tid < 256) {
            unsigned base = S.tot[tid];
            for (int u = 0; u < warp; ++u) base += (unsigned)S.wsum[u];
#pragma unroll
            for (int u = 0; u < W; ++u) S.cnt[u][tid] += base;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            if (s0 + j * 32 >= s1) continue;  // uniform over the warp
            const bool valid = s0 + j * 32 + lane < s1;
            const unsigned d = (unsigned)(w[j] >> shift) & 255u;
            const unsigned off = valid ? S.cnt[warp][d] : 0u;
            __syncwarp();
            if (valid) {
                S.s[off + (unsigned)__popc(peers[j] & lt)] = w[j];
                if ((peers[j] & lt) == 0u) S.cnt[warp][d] = off + (unsigned)__popc(peers[j]);
            }
            __syncwarp();
        }
        __syncthreads();
    }
    if (coarse) return;
    // runs of equal keys, ordered by record
    if (tid == 0) S.n_runs = 0;
    __syncthreads();
    for (int i = tid; i < n - 1; i += THREADS) {
        const unsigned k = (unsigned)(S.s[i] >> 32);
        if ((unsigned)(S.s[i + 1] >> 32) != k || (i > 0 && (unsigned)(S.s[i - 1] >> 32) == k)) continue;
        int e = i + 2;  // i starts a run of length >= 2: [i, e)
        while (e < n && e - i <= kRunSerial && (unsigned)(S.s[e] >> 32) == k) ++e;
        if (e - i > kRunSerial) {
            const int q = atomicAdd(&S.n_runs, 1);
            if (q < 64) S.runs[q] = i;
            continue;
        }
        for (int a = i + 1; a < e; ++a) {  // insertion sort by the whole word
            const unsigned long long x = S.s[a];
            int b = a - 1;
            while (b >= i && S.s[b] > x) {
                S.s[b + 1] = S.s[b];
                --b;
            }
            S.s[b + 1] = x;
        }
    }
    __syncthreads();
    const int nr = S.n_runs;
    if (nr > 64) {
        smem_sort<THREADS>(S.s, n);  // many long runs: the whole block by the full words
        return;
    }
    for (int q = 0; q < nr; ++q) {
        const int i = S.runs[q];
        const unsigned k = (unsigned)(S.s[i] >> 32);
        int e = i + 1;
        while (e < n && (unsigned)(S.s[e] >> 32) == k) ++e;  // every thread finds the same end
        smem_sort<THREADS>(S.s + i, e - i);
    }
}

// Sorts, per tile t, the words [range.x, range.y) if their count is in (lo_len, hi_len] (at most
// CAP), by the radix sort above, in shared memory. With `coarse`, only by the key's top 16 bits
// (its two upper digits) and with ties left in any order: for lists whose order only groups
// similar keys.
template <int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS) k_tile_radix(const int2 *__restrict__ ranges,
                                                        unsigned long long *__restrict__ pairs, int lo_len,
                                                        int hi_len, bool coarse) {
    extern __shared__ unsigned long long radix_raw[];
    auto &S = *reinterpret_cast<RadixSmem<CAP, THREADS> *>(radix_raw);
    const int2 rg = ranges[blockIdx.x];
    const int n = rg.y - rg.x;
    if (n <= 1 || n <= lo_len || n > hi_len || n > CAP) return;
    unsigned long long *a = pairs + rg.x;
    for (int i = threadIdx.x; i < n; i += THREADS) S.s[i] = a[i];
    __syncthreads();
    smem_radix_sort<CAP, THREADS>(S, n, coarse);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += THREADS) a[i] = S.s[i];
}

// The same radix sort for ranges longer than shared memory holds: one CTA per tile runs the four
// passes between the tile's range of `pairs` and the same range of `scratch`. The four digit
// histograms come from one read of the range; each pass is then a stable scatter of CH-word chunks
// in order (the chunk's words in registers, ranked per warp as above, placed after the words of
// earlier chunks and warps). Runs of equal keys are then ordered by record: short runs by one
// thread, long ones by the bitonic network (sort_range).
template <int THREADS, int CH>
struct RadixLongSmem {
    static constexpr int W = THREADS / 32, ITEMS = CH / THREADS, SEG = ITEMS * 32;
    unsigned cnt[W][256];
    unsigned base[256];     // per digit: the next position after the chunks placed so far
    unsigned hist[4][256];  // per pass, the digit histogram of the whole range (one read for all)
    int wsum[8];
    int skip[4];
    int n_runs;
    int runs[64];
};

template <int THREADS, int CH, int CAP>
__global__ void __launch_bounds__(THREADS) k_tile_radix_long(const int2 *__restrict__ ranges,
                                                             unsigned long long *__restrict__ pairs,
                                                             unsigned long long *__restrict__ scratch, int lo_len,
                                                             bool coarse) {
    using RS = RadixLongSmem<THREADS, CH>;
    constexpr int W = RS::W, ITEMS = RS::ITEMS, SEG = RS::SEG;
    static_assert(THREADS >= 256 && THREADS % 256 == 0, "one thread per digit in the scan");
    extern __shared__ unsigned long long radix_long_raw[];
    RS &S = *reinterpret_cast<RS *>(radix_long_raw);
    unsigned long long *bsort = radix_long_raw + (sizeof(RS) + 7) / 8;  // [CAP] for sort_range
    const int2 rg = ranges[blockIdx.x];
    const int n = rg.y - rg.x;
    if (n <= lo_len || n <= 1) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long *src = pairs + rg.x, *dst = scratch + rg.x;
    const int first_pass = coarse ? 2 : 0;
    if (tid < 4) S.skip[tid] = 0;
    for (int i = tid; i < 4 * 256; i += THREADS) (&S.hist[0][0])[i] = 0u;
    __syncthreads();
    // the histograms of every pass's digit in one read of the range (a pass moves the words, not
    // the digits' counts)
    for (int i0 = warp * 32; i0 < n; i0 += THREADS) {
        const int i = i0 + lane;
        const bool valid = i < n;
        const unsigned key = valid ? (unsigned)(src[i] >> 32) : 0u;
        const unsigned vm = __ballot_sync(0xffffffffu, valid);
        for (int pass = first_pass; pass < 4; ++pass) {
            const unsigned d = (key >> (8 * pass)) & 255u;
            unsigned m = vm;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                m &= ((d >> b) & 1u) ? bb : ~bb;
            }
            if (valid && (m & lt) == 0u) atomicAdd(&S.hist[pass][d], (unsigned)__popc(m));
        }
    }
    __syncthreads();
    for (int pass = first_pass; pass < 4; ++pass) {
        const int shift = 32 + 8 * pass;
        if (tid < 256) {
            const unsigned c = S.hist[pass][tid];
            if (c == (unsigned)n) S.skip[pass] = 1;
            unsigned inc = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (lane == 31) S.wsum[warp] = (int)inc;
            S.base[tid] = inc - c;
        }
        __syncthreads();
        if (S.skip[pass]) continue;  // uniform: nothing moves
        if (tid < 256) {
            unsigned b = S.base[tid];
            for (int u = 0; u < warp; ++u) b += (unsigned)S.wsum[u];
            S.base[tid] = b;
        }
        // chunks in order
        for (int c0 = 0; c0 < n; c0 += CH) {
            unsigned long long w[ITEMS];
            unsigned peers[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const int i = c0 + warp * SEG + j * 32 + lane;
                w[j] = i < n ? src[i] : ~0ull;
            }
            for (int d = lane; d < 256; d += 32) S.cnt[warp][d] = 0u;
            __syncwarp();
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const bool valid = c0 + warp * SEG + j * 32 + lane < n;
                const unsigned d = (unsigned)(w[j] >> shift) & 255u;
                unsigned m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
                    m &= ((d >> b) & 1u) ? bb : ~bb;
                }
                peers[j] = m;
                if (valid && (m & lt) == 0u) S.cnt[warp][d] += (unsigned)__popc(m);
                __syncwarp();
            }
            __syncthreads();  // every warp's counts (and, first chunk, the digit bases) are in
            if (tid < 256) {
                unsigned run = S.base[tid];
#pragma unroll
                for (int u = 0; u < W; ++u) {
                    const unsigned c = S.cnt[u][tid];
                    S.cnt[u][tid] = run;
                    run += c;
                }
                S.base[tid] = run;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const bool valid = c0 + warp * SEG + j * 32 + lane < n;
                const unsigned d = (unsigned)(w[j] >> shift) & 255u;
                const unsigned off = valid ? S.cnt[warp][d] : 0u;
                __syncwarp();
                if (valid) {
                    dst[off + (unsigned)__popc(peers[j] & lt)] = w[j];
                    if ((peers[j] & lt) == 0u) S.cnt[warp][d] = off + (unsigned)__popc(peers[j]);
                }
                __syncwarp();
            }
            __syncthreads();  // the counters are reused by the next chunk
        }
        __threadfence_block();
        unsigned long long *t = src;
        src = dst;
        dst = t;
    }
    // the sorted words back into `pairs` (after an odd number of moving passes they are in scratch)
    if (src != pairs + rg.x) {
        for (int i = tid; i < n; i += THREADS) pairs[rg.x + i] = src[i];
        __syncthreads();
    }
    if (coarse) return;
    unsigned long long *a = pairs + rg.x;
    if (tid == 0) S.n_runs = 0;
    __syncthreads();
    for (int i = tid; i < n - 1; i += THREADS) {
        const unsigned k = (unsigned)(a[i] >> 32);
        if ((unsigned)(a[i + 1] >> 32) != k || (i > 0 && (unsigned)(a[i - 1] >> 32) == k)) continue;
        int e = i + 2;
        while (e < n && e - i <= kRunSerial && (unsigned)(a[e] >> 32) == k) ++e;
        if (e - i > kRunSerial) {
            const int q = atomicAdd(&S.n_runs, 1);
            if (q < 64) S.runs[q] = i;
            continue;
        }
        for (int x = i + 1; x < e; ++x) {
            const unsigned long long v = a[x];
            int b = x - 1;
            while (b >= i && a[b] > v) {
                a[b + 1] = a[b];
                --b;
            }
            a[b + 1] = v;
        }
    }
    __syncthreads();
    const int nr = S.n_runs;
    if (nr > 64) {
        sort_range<CAP, THREADS>(a, n, bsort);
        return;
    }
    for (int q = 0; q < nr; ++q) {
        const int i = S.runs[q];
        const unsigned k = (unsigned)(a[i] >> 32);
        int e = i + 1;
        while (e < n && (unsigned)(a[e] >> 32) == k) ++e;
        sort_range<CAP, THREADS>(a + i, e - i, bsort);
        __syncthreads();
    }
}

// Sorts, per tile t, the words [range.x, end[t]) (default end: range.y) if their count is in
// (lo_len, hi_len]; with blocks_only, each CAP-word block of a longer range on its own.
template <int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS) k_tile_sort(const int2 *__restrict__ ranges, const int *__restrict__ end,
                                                       unsigned long long *__restrict__ pairs, int lo_len, int hi_len,
                                                       bool blocks_only) {
    extern __shared__ unsigned long long s[];  // [CAP]
    const int2 rg = ranges[blockIdx.x];
    const int y = end ? end[blockIdx.x] : rg.y;
    const int n = y - rg.x;
    if (n <= 1 || n <= lo_len || n > hi_len) return;
    sort_range<CAP, THREADS>(pairs + rg.x, n, s, blocks_only);
}

// Sorts the rest of the lists of the tiles in list[0, *count): [prefix_end[t], range.y). A fixed
// grid walks the list, which the composite fills on the device.
template <int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS) k_tail_sort(const int2 *__restrict__ ranges,
                                                       const int *__restrict__ prefix_end, const int *__restrict__ list,
                                                       const int *__restrict__ count, unsigned long long *__restrict__ pairs) {
    extern __shared__ unsigned long long s[];  // [CAP]
    const int nt = *count;
    for (int i = blockIdx.x; i < nt; i += gridDim.x) {
        const int t = list[i];
        const int x = prefix_end[t];
        sort_range<CAP, THREADS>(pairs + x, ranges[t].y - x, s);
        __syncthreads();
    }
}

constexpr int kSelBins = 2048;  // 11 key bits per histogram level

// Smallest bin b of hist[kSelBins] with (count of bins <= b) >= need (1 <= need <= total):
// out[0] = b, out[1] = count of the bins below b.
template <int THREADS>
__device__ void find_bin(const int *hist, int need, int *warp_tot, int *out) {
    constexpr int PER = kSelBins / THREADS;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int loc[PER], sum = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        loc[i] = hist[tid * PER + i];
        sum += loc[i];
    }
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    int ex = inc - sum;
    for (int u = 0; u < w; ++u) ex += warp_tot[u];
    if (ex < need && need <= ex + sum) {
        int c = ex;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if (c + loc[i] >= need) {
                out[0] = tid * PER + i;
                out[1] = c;
                break;
            }
            c += loc[i];
        }
    }
    __syncthreads();
}

// Front selection and sort of one tile (see the top of the file). The tile's bucketed words are
// read from `in` and its list is written to `out`: the sorted front, then the rest. A list of at
// most prefix * 3 / 2 words is sorted whole. Fronts or whole lists longer than CAP are copied
// unsorted and left to the long-list sort, which sorts [range.x, prefix_end).
template <int CAP, int THREADS>
__global__ void __launch_bounds__(THREADS) k_tile_select(const int2 *__restrict__ ranges,
                                                         const unsigned long long *__restrict__ in,
                                                         unsigned long long *__restrict__ out, int prefix,
                                                         int *__restrict__ prefix_end, float *__restrict__ prefix_key,
                                                         int *__restrict__ tile_flag) {
    extern __shared__ unsigned long long s[];  // [CAP]
    __shared__ int hist[kSelBins];
    __shared__ int warp_tot[THREADS / 32];
    __shared__ int sel[4];  // bin, words below it, front cursor, rest cursor
    const int t = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
    const int2 rg = ranges[t];
    const int n = rg.y - rg.x;
    const unsigned long long *a = in + rg.x;
    unsigned long long *o = out + rg.x;
    if (tid == 0) tile_flag[t] = 0;
    int F = n;
    unsigned thr = 0;  // the front: words with key >> 9 <= thr
    if (prefix > 0 && n > prefix + prefix / 2) {
        // level 1: key bits 30..20 (the sign bit of a depth key is 0)
        for (int i = tid; i < kSelBins; i += THREADS) hist[i] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += THREADS) atomicAdd(&hist[(unsigned)(a[i] >> 52)], 1);
        __syncthreads();
        find_bin<THREADS>(hist, prefix, warp_tot, sel);
        const unsigned b1 = (unsigned)sel[0];
        const int before = sel[1];
        F = before + hist[b1];
        thr = (b1 << 11) | 2047u;
        if (F > CAP) {
            // level 2 inside bin b1: key bits 19..9
            __syncthreads();
            for (int i = tid; i < kSelBins; i += THREADS) hist[i] = 0;
            __syncthreads();
            for (int i = tid; i < n; i += THREADS) {
                const unsigned long long w = a[i];
                if ((unsigned)(w >> 52) == b1) atomicAdd(&hist[(unsigned)(w >> 41) & 2047u], 1);
            }
            __syncthreads();
            find_bin<THREADS>(hist, prefix - before, warp_tot, sel);
            F = before + sel[1] + hist[sel[0]];
            thr = (b1 << 11) | (unsigned)sel[0];
        }
    }
    if (F >= n) {
        // the whole list
        if (tid == 0) {
            prefix_end[t] = rg.y;
            prefix_key[t] = INFINITY;
        }
        if (n > CAP) {
            for (int i = tid; i < n; i += THREADS) o[i] = a[i];
            return;
        }
        for (int i = tid; i < n; i += THREADS) s[i] = a[i];
        __syncthreads();
        smem_sort<THREADS>(s, n);
        for (int i = tid; i < n; i += THREADS) o[i] = s[i];
        return;
    }
    // partition: the front into shared memory (or `out` if longer than CAP), the rest after it
    if (tid == 0) {
        sel[2] = 0;
        sel[3] = 0;
        prefix_end[t] = rg.x + F;
        prefix_key[t] = __uint_as_float((thr + 1u) << 9);  // every key of the rest is >= this
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int i0 = 0; i0 < n; i0 += THREADS) {
        const int i = i0 + tid;
        const bool v = i < n;
        const unsigned long long w = v ? a[i] : 0ull;
        const bool f = v && (unsigned)(w >> 41) <= thr;
        const unsigned fm = __ballot_sync(0xffffffffu, f), rm = __ballot_sync(0xffffffffu, v && !f);
        int fb = 0, rb = 0;
        if (lane == 0) {
            if (fm) fb = atomicAdd(&sel[2], __popc(fm));
            if (rm) rb = atomicAdd(&sel[3], __popc(rm));
        }
        fb = __shfl_sync(0xffffffffu, fb, 0);
        rb = __shfl_sync(0xffffffffu, rb, 0);
        if (f) {
            const int q = fb + __popc(fm & lt);
            if (F <= CAP)
                s[q] = w;
            else
                o[q] = w;
        } else if (v) {
            o[F + rb + __popc(rm & lt)] = w;
        }
    }
    if (F > CAP) return;
    __syncthreads();
    smem_sort<THREADS>(s, F);
    for (int i = tid; i < F; i += THREADS) o[i] = s[i];
}

}  // namespace

// the long-list radix sort: 4096-word chunks, and a 4096-word block for its bitonic fallback
constexpr int kLongChunk = 4096;
constexpr size_t kLongSmem =
    (sizeof(RadixLongSmem<kLargeThreads, kLongChunk>) + 7) / 8 * 8 + (size_t)kSmallCap * sizeof(unsigned long long);

template <int CAP, int THREADS>
cudaError_t set_smem(const void *fn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(CAP * sizeof(unsigned long long)));
}

cudaError_t launch_tile_buckets(const unsigned *ptile, const unsigned *pkey, const unsigned *prec,
                                const unsigned long long *n_dev, long long cap, const int *tile_counts,
                                const int *tile_offsets, int n_tiles, int2 *ranges, int *cursor,
                                unsigned long long *pairs, unsigned long long *pair_total, cudaStream_t s,
                                const FrontSort *front, bool blocks_only, unsigned long long *scratch,
                                const unsigned *prank) {
    if (n_tiles <= 0) return cudaSuccess;
    note_launches(3);
    k_ranges_from_counts<<<(n_tiles + 255) / 256, 256, 0, s>>>(tile_counts, tile_offsets, n_tiles, ranges, cursor);
    if (cap > 0)
        k_bucket<<<(unsigned)((cap + 255) / 256), 256, 0, s>>>(ptile, pkey, prec, n_dev, cap, cursor, pairs,
                                                               pair_total, prank, tile_offsets);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = set_smem<kLargeCap, kLargeThreads>((const void *)k_tile_sort<kLargeCap, kLargeThreads>);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    constexpr size_t small_sm = kSmallCap * sizeof(unsigned long long);
    constexpr size_t large_sm = kLargeCap * sizeof(unsigned long long);
    note_launches(1);
    if (!front) {
        // in place, whole lists: up to kLargeCap words by the radix sort in shared memory, longer
        // ones by the bitonic network with its exchanges at distance >= kLargeCap in global memory
        static bool radix_configured = false;
        using SmallRadix = RadixSmem<kSmallCap, kSmallThreads>;
        using LargeRadix = RadixSmem<kLargeCap, kLargeThreads>;
        if (!radix_configured) {
            cudaError_t e = cudaFuncSetAttribute((const void *)k_tile_radix<kSmallCap, kSmallThreads>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmallRadix));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute((const void *)k_tile_radix<kLargeCap, kLargeThreads>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LargeRadix));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute((const void *)k_tile_radix_long<kLargeThreads, kLongChunk, kSmallCap>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLongSmem);
            if (e != cudaSuccess) return e;
            radix_configured = true;
        }
        note_launches(1);  // the third sort launch
        k_tile_radix<kSmallCap, kSmallThreads><<<n_tiles, kSmallThreads, sizeof(SmallRadix), s>>>(
            ranges, pairs, 0, kSmallCap, blocks_only);
        k_tile_radix<kLargeCap, kLargeThreads><<<n_tiles, kLargeThreads, sizeof(LargeRadix), s>>>(
            ranges, pairs, kSmallCap, kLargeCap, blocks_only);
        if (scratch) {
            k_tile_radix_long<kLargeThreads, kLongChunk, kSmallCap><<<n_tiles, kLargeThreads, kLongSmem, s>>>(
                ranges, pairs, scratch, kLargeCap, blocks_only);
        } else {
            k_tile_sort<kLargeCap, kLargeThreads><<<n_tiles, kLargeThreads, large_sm, s>>>(
                ranges, nullptr, pairs, kLargeCap, 1 << 30, blocks_only);
        }
        return cudaGetLastError();
    }
    k_tile_select<kSmallCap, kSmallThreads><<<n_tiles, kSmallThreads, small_sm, s>>>(
        ranges, pairs, front->out, front->prefix, front->prefix_end, front->prefix_key, front->tile_flag);
    k_tile_sort<kLargeCap, kLargeThreads><<<n_tiles, kLargeThreads, large_sm, s>>>(ranges, front->prefix_end,
                                                                                  front->out, kSmallCap, 1 << 30, false);
    return cudaGetLastError();
}

// The rest of the lists of the tiles in list[0, *count).
cudaError_t launch_tail_sort(const int2 *ranges, const int *prefix_end, const int *list, const int *count,
                             unsigned long long *pairs, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = set_smem<kLargeCap, kLargeThreads>((const void *)k_tail_sort<kLargeCap, kLargeThreads>);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    note_launches(1);
    k_tail_sort<kLargeCap, kLargeThreads><<<device_sm_count() * 2, kLargeThreads, kLargeCap * sizeof(unsigned long long), s>>>(
        ranges, prefix_end, list, count, pairs);
    return cudaGetLastError();
}

}  // namespace sof
