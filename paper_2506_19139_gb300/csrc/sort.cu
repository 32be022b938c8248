// LSD radix sort of (64-bit key, 32-bit value) pairs over a bit range, 8-bit digits, stable.
// Per pass: k_digit_hist (per-block digit histograms, digit-major), a device exclusive scan of
// the histograms, and k_digit_scatter, which ranks each item among equal digits of its block in
// input order (warp match + per-warp counters) and writes it to its global position.
// Also k_tile_ranges, which turns the sorted keys into [start, end) runs per global tile.
#include "sof_internal.cuh"

namespace sof {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                          // per thread
constexpr int kSortTile = kSortThreads * kSortItems;    // 4096 items per block
constexpr int kWarpTile = 32 * kSortItems;              // 512 consecutive items per warp

__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const unsigned long long *__restrict__ keys,
                                                             long long n, int shift, int n_blocks,
                                                             int *__restrict__ hist) {
    __shared__ int h[kSortWarps][256];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kSortTile + (long long)w * kWarpTile;
#pragma unroll 4
    for (int r = 0; r < kSortItems; ++r) {
        long long i = base + r * 32 + lane;
        if (i < n) atomicAdd(&h[w][(int)((keys[i] >> shift) & 0xFFu)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += kSortThreads) {
        int s = 0;
#pragma unroll
        for (int k = 0; k < kSortWarps; ++k) s += h[k][d];
        hist[(long long)d * n_blocks + blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(kSortThreads) k_digit_scatter(const unsigned long long *__restrict__ keys_in,
                                                                const unsigned *__restrict__ vals_in,
                                                                unsigned long long *__restrict__ keys_out,
                                                                unsigned *__restrict__ vals_out, long long n,
                                                                int shift, int n_blocks,
                                                                const int *__restrict__ offsets) {
    __shared__ int wcnt[kSortWarps][256];
    __shared__ int gofs[256];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    for (int d = threadIdx.x; d < 256; d += kSortThreads) gofs[d] = offsets[(long long)d * n_blocks + blockIdx.x];
    __syncthreads();
    long long base = (long long)blockIdx.x * kSortTile + (long long)w * kWarpTile;
    unsigned long long k[kSortItems];
    unsigned v[kSortItems];
    int local[kSortItems];
    unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        long long i = base + r * 32 + lane;
        bool valid = i < n;
        k[r] = valid ? keys_in[i] : 0ull;
        v[r] = valid ? vals_in[i] : 0u;
        int d = valid ? (int)((k[r] >> shift) & 0xFFu) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        int leader = __ffs(peers) - 1;
        int before = valid ? wcnt[w][d] : 0;
        __syncwarp();
        if (valid && lane == leader) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        local[r] = before + rank;
    }
    __syncthreads();
    // exclusive scan over warps per digit
    for (int d = threadIdx.x; d < 256; d += kSortThreads) {
        int run = 0;
#pragma unroll
        for (int q = 0; q < kSortWarps; ++q) {
            int c = wcnt[q][d];
            wcnt[q][d] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        long long i = base + r * 32 + lane;
        if (i < n) {
            int d = (int)((k[r] >> shift) & 0xFFu);
            long long pos = (long long)gofs[d] + wcnt[w][d] + local[r];
            keys_out[pos] = k[r];
            vals_out[pos] = v[r];
        }
    }
}

__global__ void k_tile_ranges(const unsigned long long *__restrict__ keys, long long n, int2 *__restrict__ ranges,
                              int n_tiles) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned t = (unsigned)(keys[i] >> 32);
    if ((int)t >= n_tiles) return;
    if (i == 0 || (unsigned)(keys[i - 1] >> 32) != t) ranges[t].x = (int)i;
    if (i == n - 1 || (unsigned)(keys[i + 1] >> 32) != t) ranges[t].y = (int)(i + 1);
}

long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

}  // namespace

size_t radix_sort_temp_bytes(long long n) {
    long long blocks = cdiv(n > 0 ? n : 1, kSortTile);
    size_t hist = ((size_t)blocks * 256 * sizeof(int) + 255) / 256 * 256;
    return 2 * hist + scan_temp_bytes(blocks * 256) + 256;
}

cudaError_t radix_sort_pairs(unsigned long long *keys, unsigned *vals, unsigned long long *keys_alt,
                             unsigned *vals_alt, long long n, int begin_bit, int end_bit, void *temp,
                             bool *result_in_alt, cudaStream_t s) {
    *result_in_alt = false;
    if (n <= 1) return cudaSuccess;
    long long blocks = cdiv(n, kSortTile);
    size_t hist_bytes = ((size_t)blocks * 256 * sizeof(int) + 255) / 256 * 256;
    int *hist = reinterpret_cast<int *>(temp);
    int *offs = reinterpret_cast<int *>(reinterpret_cast<char *>(temp) + hist_bytes);
    void *scan_tmp = reinterpret_cast<char *>(temp) + 2 * hist_bytes;
    unsigned long long *kin = keys, *kout = keys_alt;
    unsigned *vin = vals, *vout = vals_alt;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        note_launches(1);
        k_digit_hist<<<(unsigned)blocks, kSortThreads, 0, s>>>(kin, n, shift, (int)blocks, hist);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_exclusive_scan(hist, offs, blocks * 256, scan_tmp, nullptr, s);
        if (e != cudaSuccess) return e;
        note_launches(1);
        k_digit_scatter<<<(unsigned)blocks, kSortThreads, 0, s>>>(kin, vin, kout, vout, n, shift, (int)blocks, offs);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        unsigned long long *tk = kin; kin = kout; kout = tk;
        unsigned *tv = vin; vin = vout; vout = tv;
        *result_in_alt = !*result_in_alt;
    }
    return cudaSuccess;
}

cudaError_t launch_tile_ranges(const unsigned long long *keys, long long n, int2 *ranges, int n_tiles,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    note_launches(1);
    k_tile_ranges<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(keys, n, ranges, n_tiles);
    return cudaGetLastError();
}

}  // namespace sof
