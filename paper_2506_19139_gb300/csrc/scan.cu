// Device-wide exclusive prefix sum of int32 counts (recursive, 2048 items per block).
#include "sof_internal.cuh"

namespace sof {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int x, int *warp_tot, int *block_total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        int t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
        int ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;
        if (lane == kScanThreads / 32 - 1) *block_total = ti;
    }
    __syncthreads();
    return warp_tot[w] + inc - x;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int *__restrict__ in, int *__restrict__ out,
                                                             long long n, int *__restrict__ tile_sums) {
    __shared__ int warp_tot[kScanThreads / 32];
    __shared__ int total;
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int ex = block_exclusive_scan(s, warp_tot, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(int *__restrict__ out, long long n,
                                                           const int *__restrict__ tile_offsets) {
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int add = tile_offsets[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) out[base + i] += add;
}

// total = out[n-1] + in[n-1]
__global__ void k_scan_total(const int *in, const int *out, long long n, int *total) {
    *total = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

}  // namespace

size_t scan_temp_bytes(long long n) {
    size_t bytes = 0;
    while (n > kScanTile) {
        n = ceil_div(n, kScanTile);
        bytes += 2 * ((size_t)n * sizeof(int) + 256);
    }
    return bytes + 256;
}

static cudaError_t scan_rec(const int *in, int *out, long long n, char *temp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long tiles = ceil_div(n, kScanTile);
    if (tiles == 1) {
        note_launches(1);
        k_scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        return cudaGetLastError();
    }
    int *sums = reinterpret_cast<int *>(temp);
    int *sums_scan = reinterpret_cast<int *>(temp + ((tiles * sizeof(int) + 255) / 256) * 256);
    char *next = temp + 2 * (((tiles * sizeof(int) + 255) / 256) * 256);
    note_launches(1);
    k_scan_tiles<<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_rec(sums, sums_scan, tiles, next, s);
    if (e != cudaSuccess) return e;
    note_launches(1);
    k_scan_add<<<(unsigned)tiles, kScanThreads, 0, s>>>(out, n, sums_scan);
    return cudaGetLastError();
}

cudaError_t launch_exclusive_scan(const int *in, int *out, long long n, void *temp, int *total_dev,
                                  cudaStream_t s) {
    cudaError_t e = scan_rec(in, out, n, reinterpret_cast<char *>(temp), s);
    if (e != cudaSuccess) return e;
    if (total_dev) {
        note_launches(1);
        k_scan_total<<<1, 1, 0, s>>>(in, out, n, total_dev);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace sof
