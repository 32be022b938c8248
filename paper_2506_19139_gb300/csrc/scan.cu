// Device-wide exclusive prefix sum of int32 counts into int32 or int64 sums (recursive, 2048 items
// per block).
#include <stddef.h>
#include <stdint.h>

#include "sof_internal.cuh"

namespace sof {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T x, T *warp_tot, T *block_total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    if (w == 0) {
        T t = lane < kScanThreads / 32 ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;
        if (lane == kScanThreads / 32 - 1) *block_total = ti;
    }
    __syncthreads();
    return warp_tot[w] + inc - x;
}

// TI: the counts' type, TO: the sums' (int, or long long where the total may pass 2^31)
template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const TI *__restrict__ in, TO *__restrict__ out,
                                                             long long n, TO *__restrict__ tile_sums) {
    __shared__ TO warp_tot[kScanThreads / 32];
    __shared__ TO total;
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    TO v[kScanItems];
    TO s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? (TO)in[base + i] : TO(0);
        s += v[i];
    }
    TO ex = block_exclusive_scan<TO>(s, warp_tot, &total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = total;
}

template <typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_add(TO *__restrict__ out, long long n,
                                                           const TO *__restrict__ tile_offsets) {
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    TO add = tile_offsets[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) out[base + i] += add;
}

// total = out[n-1] + in[n-1]
template <typename TI, typename TO>
__global__ void k_scan_total(const TI *in, const TO *out, long long n, TO *total) {
    *total = n > 0 ? out[n - 1] + (TO)in[n - 1] : TO(0);
}

long long ceil_div(long long a, long long b) { return (a + b - 1) / b; }

}  // namespace

size_t scan_temp_bytes(long long n) {
    size_t bytes = 0;
    while (n > kScanTile) {
        n = ceil_div(n, kScanTile);
        bytes += 2 * ((size_t)n * sizeof(long long) + 256);
    }
    return bytes + 256;
}

template <typename TI, typename TO>
static cudaError_t scan_rec(const TI *in, TO *out, long long n, char *temp, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long tiles = ceil_div(n, kScanTile);
    if (tiles == 1) {
        note_launches(1);
        k_scan_tiles<TI, TO><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
        return cudaGetLastError();
    }
    TO *sums = reinterpret_cast<TO *>(temp);
    TO *sums_scan = reinterpret_cast<TO *>(temp + ((tiles * sizeof(TO) + 255) / 256) * 256);
    char *next = temp + 2 * (((tiles * sizeof(TO) + 255) / 256) * 256);
    note_launches(1);
    k_scan_tiles<TI, TO><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_rec<TO, TO>(sums, sums_scan, tiles, next, s);
    if (e != cudaSuccess) return e;
    note_launches(1);
    k_scan_add<TO><<<(unsigned)tiles, kScanThreads, 0, s>>>(out, n, sums_scan);
    return cudaGetLastError();
}

cudaError_t launch_exclusive_scan(const int *in, int *out, long long n, void *temp, int *total_dev,
                                  cudaStream_t s) {
    cudaError_t e = scan_rec<int, int>(in, out, n, reinterpret_cast<char *>(temp), s);
    if (e != cudaSuccess) return e;
    if (total_dev) {
        note_launches(1);
        k_scan_total<int, int><<<1, 1, 0, s>>>(in, out, n, total_dev);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_exclusive_scan64(const int *in, long long *out, long long n, void *temp, long long *total_dev,
                                    cudaStream_t s) {
    cudaError_t e = scan_rec<int, long long>(in, out, n, reinterpret_cast<char *>(temp), s);
    if (e != cudaSuccess) return e;
    if (total_dev) {
        note_launches(1);
        k_scan_total<int, long long><<<1, 1, 0, s>>>(in, out, n, total_dev);
        e = cudaGetLastError();
    }
    return e;
}

namespace {
// 64-bit sum of n int32 values into *acc (one atomic per block): detects totals that the int32
// scan cannot represent.
__global__ void __launch_bounds__(kScanThreads) k_sum64(const int *__restrict__ in, long long n,
                                                        unsigned long long *__restrict__ acc) {
    __shared__ unsigned long long part[kScanThreads / 32];
    unsigned long long s = 0;
    const long long base = (long long)blockIdx.x * kScanTile + threadIdx.x;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long k = base + (long long)i * kScanThreads;
        if (k < n) s += (unsigned long long)(unsigned)in[k];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += part[w];
        if (t) atomicAdd(acc, t);
    }
}

__global__ void k_set_cams(const CamSet cams, int n_words, unsigned *__restrict__ dst) {
    const unsigned *src = reinterpret_cast<const unsigned *>(&cams);
    for (int i = threadIdx.x; i < n_words; i += blockDim.x) dst[i] = src[i];
}
}  // namespace

cudaError_t launch_sum64(const int *in, long long n, unsigned long long *acc, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    note_launches(1);
    k_sum64<<<(unsigned)ceil_div(n, kScanTile), kScanThreads, 0, s>>>(in, n, acc);
    return cudaGetLastError();
}

namespace {
__global__ void k_guard_items(const unsigned long long *area_total, int *n_items, unsigned long long *dropped) {
    if (*area_total > (unsigned long long)INT32_MAX - 1024) {
        atomicAdd(dropped, *area_total);
        *n_items = 0;
    }
}
}  // namespace

// Without a host round trip: a pair bound beyond 32-bit indexing voids the call (all counted as
// dropped) instead of binning with a wrapped count.
cudaError_t launch_guard_items(const unsigned long long *area_total, int *n_items, unsigned long long *dropped,
                               cudaStream_t s) {
    note_launches(1);
    k_guard_items<<<1, 1, 0, s>>>(area_total, n_items, dropped);
    return cudaGetLastError();
}

namespace {
__global__ void k_add_u64(const unsigned long long *src, unsigned long long *dst) { *dst += *src; }
}  // namespace

cudaError_t launch_add_u64(const unsigned long long *src, unsigned long long *dst, cudaStream_t s) {
    note_launches(1);
    k_add_u64<<<1, 1, 0, s>>>(src, dst);
    return cudaGetLastError();
}

int device_sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return 152;  // GB300 has 152 SMs; only reached when the device cannot be named
    }
    if (cached[dev] <= 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 152;
        }
        cached[dev] = n;
    }
    return cached[dev];
}

cudaError_t launch_set_cams(const CamSet &cams, CamSet *dst, cudaStream_t s) {
    const size_t bytes = offsetof(CamSet, cam) + (size_t)cams.n_views * sizeof(DevCam);
    note_launches(1);
    k_set_cams<<<1, 256, 0, s>>>(cams, (int)((bytes + 3) / 4), reinterpret_cast<unsigned *>(dst));
    return cudaGetLastError();
}

}  // namespace sof
