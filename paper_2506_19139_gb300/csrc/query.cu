// Opacity field at 3D points, min over views (Eqs. 11-12, App. A.2; Sec. 3.4 "Ray/Tile
// Scheduling", "Early Stopping").
//
// Per view: the Gaussians are bucketed by screen tile and sorted by z_min within each tile (one
// word z_min bits << 32 | record), z_min the exact minimum camera z of the E-ellipsoid; the visible
// points are bucketed by tile and grouped by camera z (z bits << 32 | point, sorted within blocks of
// 8192), so that each CTA of 256 threads takes up to 256 points of one tile at similar depths (a
// block -> tile table, as in the paper's scheduling). Each thread evaluates one point
// against the tile's Gaussians in z_min order and stops at the first with z_min > z(point): no
// later one can reach alpha >= 1/255 at t_eval <= t. O_N = 1 - prod(1 - alpha) needs no order
// (App. A.2). A view's running value only grows, so a thread also stops once it reaches the
// point's current minimum over the views already done (exact pruning; the min cannot change).
#include <math.h>

#include "record.cuh"
#include "sof_internal.cuh"

namespace sof {
namespace {

constexpr int kQThreads = 256;
constexpr int kQChunk = 64;

struct PointProj {
    bool vis;
    float Xh, Xl, Yh, Yl, zh, zl, dn;
    int px, py;
};

// Camera-space position in FP64 (FP32 products are exact), projection split into hi + lo floats.
__device__ __forceinline__ PointProj project_point(const DevCam &cam, const float *pts, long long i, float near_plane) {
    PointProj r;
    double x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    double xc = cam.R[0] * x + cam.R[1] * y + cam.R[2] * z + cam.t[0];
    double yc = cam.R[3] * x + cam.R[4] * y + cam.R[5] * z + cam.t[1];
    double zc = cam.R[6] * x + cam.R[7] * y + cam.R[8] * z + cam.t[2];
    r.vis = false;
    r.px = r.py = 0;
    r.Xh = r.Xl = r.Yh = r.Yl = r.zh = r.zl = r.dn = 0.f;
    if (!(zc > (double)near_plane)) return r;
    const double iz = recip_fp64(zc);
    double u = xc * iz, v = yc * iz;
    double X = (double)cam.fx * u + (double)cam.cx, Y = (double)cam.fy * v + (double)cam.cy;
    if (!(X >= 0.0 && X < (double)cam.W && Y >= 0.0 && Y < (double)cam.H)) return r;
    r.vis = true;
    r.Xh = (float)X; r.Xl = (float)(X - (double)r.Xh);
    r.Yh = (float)Y; r.Yl = (float)(Y - (double)r.Yh);
    r.zh = (float)zc; r.zl = (float)(zc - (double)r.zh);
    r.dn = sqrtf((float)(1.0 + u * u + v * v));  // |d'|, an FP32 value: a float root suffices
    r.px = min((int)X, cam.W - 1);
    r.py = min((int)Y, cam.H - 1);
    return r;
}

// Projects every point into the view; a visible one is counted in seen[], counted in its tile and
// appended, at a warp-reserved position, to an unsorted list (tile, z bits, point).
__global__ void __launch_bounds__(256) k_point_append(const CamSet *__restrict__ cams, int view,
                                                      const float *__restrict__ pts, long long n_points,
                                                      float near_plane, int *__restrict__ seen,
                                                      int *__restrict__ cursor, unsigned *__restrict__ ptile,
                                                      unsigned *__restrict__ pkey, unsigned *__restrict__ pidx,
                                                      int *__restrict__ tile_counts) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const DevCam &cam = cams->cam[view];
    bool vis = false;
    unsigned gt = 0u, key = 0u;
    if (i < n_points) {
        const PointProj pp = project_point(cam, pts, i, near_plane);
        vis = pp.vis;
        if (vis) {
            const int tile = cams->tile;
            gt = (unsigned)(cam.tile_base + (pp.py / tile) * cam.tiles_x + pp.px / tile);
            key = __float_as_uint(pp.zh);  // z > near > 0: the bits order like the values
            if (seen) seen[i] += 1;
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, vis);
    if (m == 0u) return;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0) base = atomicAdd(cursor, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (vis) {
        const int pos = base + __popc(m & ((1u << lane) - 1u));
        ptile[pos] = gt;
        pkey[pos] = key;
        pidx[pos] = (unsigned)i;
        atomicAdd(&tile_counts[gt], 1);
    }
}

// Blocks of kQThreads points per tile: nb[t] = ceil(points in t / kQThreads).
__global__ void k_tile_blocks(const int *__restrict__ pcounts, int n_tiles, int *__restrict__ nb) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    nb[t] = (pcounts[t] + kQThreads - 1) / kQThreads;
}

__global__ void k_fill_lut(const int *__restrict__ nb, const int *__restrict__ bstart, int n_tiles, int2 *__restrict__ lut) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tiles) return;
    int s = bstart[t], k = nb[t];
    for (int b = 0; b < k; ++b) lut[s + b] = make_int2(t, b);
}

__global__ void __launch_bounds__(kQThreads) k_integrate(const CamSet *__restrict__ cams, int view,
                                                         const float4 *__restrict__ qrec,
                                                         const unsigned long long *__restrict__ gpairs,
                                                         const int2 *__restrict__ granges,
                                                         const unsigned long long *__restrict__ ppairs,
                                                         const int2 *__restrict__ pranges,
                                                         const int2 *__restrict__ lut, const int *__restrict__ n_blocks,
                                                         const float *__restrict__ pts, float near_plane, float t_stop,
                                                         bool level_set, float *__restrict__ opacity_out,
                                                         DevStatus *status) {
    __shared__ float4 srec[7][kQChunk];
    __shared__ float szmin[kQChunk];
    __shared__ float sproj[kQChunk];
    const int tid = threadIdx.x;
    if ((int)blockIdx.x >= *n_blocks) return;  // the grid is sized for the most blocks a view can need
    const int2 tb = lut[blockIdx.x];
    const int2 pr = pranges[tb.x];
    const int p0 = pr.x + tb.y * kQThreads;
    const int np = min(kQThreads, pr.y - p0);
    const DevCam &cam = cams->cam[view];
    const int2 gr = granges[tb.x];
    bool done = tid >= np;
    long long pi = 0;
    PointProj pp;
    pp.vis = false;
    float P = 1.f, stop_at = 0.f;
    unsigned n_tests = 0, n_inc = 0;
    if (!done) {
        pi = (unsigned)ppairs[p0 + tid];
        pp = project_point(cam, pts, pi, near_plane);
        const float cur = opacity_out[pi];  // running min over the views done so far
        // stop once 1 - P >= cur (this view cannot lower the min any more), P < t_stop, or
        // P <= 2^-25: from there on 1 - P rounds to 1.0f whatever is multiplied in, so stopping
        // leaves the FP32 result unchanged
        stop_at = fmaxf(fmaxf(1.f - cur, t_stop), 0x1p-25f);
        done = !pp.vis || cur <= 0.f;
        if (level_set) {
            // only O > 0.5 matters: this view is done once 1 - P > 0.5 (P below 0.5, the largest
            // float under 0.5 being 0.5 - 2^-25), and a point some view left at O <= 0.5 is out
            stop_at = fmaxf(stop_at, 0.5f - 0x1p-25f);
            done = done || cur <= 0.5f;
        }
    }
    for (int base = gr.x; base < gr.y; base += kQChunk) {
        const int n = min(kQChunk, gr.y - base);
        __syncthreads();
        for (int i = tid; i < n * 7; i += kQThreads) {
            const int j = i / 7, f = i - j * 7;
            srec[f][j] = qrec[(size_t)(unsigned)gpairs[base + j] * kRecF4 + f];
        }
        for (int i = tid; i < n; i += kQThreads) {
            const unsigned long long w = gpairs[base + i];
            szmin[i] = __uint_as_float((unsigned)(w >> 32));
            sproj[i] = qrec[(size_t)(unsigned)w * kRecF4 + 7].y;
        }
        __syncthreads();
        if (!done) {
            for (int j = 0; j < n; ++j) {
                if (szmin[j] > pp.zh) {  // z_min order: no later Gaussian can contribute
                    done = true;
                    break;
                }
                const float4 r0 = srec[0][j], r2 = srec[2][j], r3 = srec[3][j], r4 = srec[4][j], r5 = srec[5][j];
                // offset from the anchor pixel centre (ia + 0.5, ja + 0.5), cancellation-free
                const float dx = (pp.Xh - (r0.x + 0.5f)) + pp.Xl;
                const float dy = (pp.Yh - (r0.y + 0.5f)) + pp.Yl;
                const RecEval e = rec_eval(r0, srec[1][j], r2, r3, r4, r5, dx, dy);
                ++n_tests;
                if (!(e.N <= __fmul_rn(r0.z, e.A))) continue;  // the line misses the E-ellipsoid
                const float rA = __frcp_rn(e.A);
                const float m = __fmul_rn(e.N, rA);
                float tstar, behind;  // peak t*' (camera-z units) and z(point) - t*'
                if (sproj[j] != 0.f) {
                    const float4 r6 = srec[6][j];
                    // z_mu - t*' = z_mu d_g . ((dx + delta_x) a + (dy + delta_y) b) / A
                    const float ex_ = dx + r6.x, ey_ = dy + r6.y;
                    const float vx = fmaf(ey_, r4.z, ex_ * r3.w);
                    const float vy = fmaf(ey_, r4.w, ex_ * r4.x);
                    const float vz = fmaf(ey_, r5.x, ex_ * r4.y);
                    const float poly = fmaf(e.gx, vx, fmaf(e.gy, vy, e.gz * vz));
                    const float zmu = r6.z + r6.w;
                    const float rel = zmu * poly * rA;
                    tstar = zmu - rel;
                    behind = ((pp.zh - r6.z) + (pp.zl - r6.w)) + rel;
                } else {
                    tstar = -rec_od(r2, dx, dy) * rA;
                    behind = (pp.zh - tstar) + pp.zl;
                }
                const float ex = behind >= 0.f ? m : fmaf(e.A * behind, behind, m);
                const float a = fminf(kAlphaMax, r0.w * __expf(-0.5f * ex));
                if (a >= kAlphaMin && tstar * pp.dn > near_plane) {
                    ++n_inc;
                    P *= (1.f - a);
                    if (P <= stop_at) {
                        done = true;
                        break;
                    }
                }
            }
        }
        if (__syncthreads_and(done)) break;
    }
    if (tid < np && pp.vis) {
        float O = 1.f - P;
        if (O < opacity_out[pi]) atomicMin(reinterpret_cast<int *>(opacity_out + pi), __float_as_int(O));
    }
    if (tid == 0) add_count(status, kCntPointViews, (unsigned long long)np);
    // work counters: one atomic per warp
    unsigned long long a = n_tests, b = n_inc;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((tid & 31) == 0 && a) {
        add_count(status, kCntTests, a);
        add_count(status, kCntHits, b);
    }
}

__global__ void k_fill(float *p, long long n, float v) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

cudaError_t launch_fill(float *p, long long n, float v, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    note_launches(1);
    k_fill<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_point_append(const CamSet *cams_dev, int view, const float *pts, long long n_points,
                               float near_plane, int *seen, int *cursor, unsigned *ptile, unsigned *pkey,
                               unsigned *pidx, int *tile_counts, cudaStream_t s) {
    if (n_points <= 0) return cudaSuccess;
    note_launches(1);
    k_point_append<<<(unsigned)((n_points + 255) / 256), 256, 0, s>>>(cams_dev, view, pts, n_points, near_plane, seen,
                                                                       cursor, ptile, pkey, pidx, tile_counts);
    return cudaGetLastError();
}

cudaError_t launch_tile_blocks(const int *pcounts, int n_tiles, int *nb, cudaStream_t s) {
    note_launches(1);
    k_tile_blocks<<<(n_tiles + 255) / 256, 256, 0, s>>>(pcounts, n_tiles, nb);
    return cudaGetLastError();
}

cudaError_t launch_fill_lut(const int *nb, const int *bstart, int n_tiles, int2 *lut, cudaStream_t s) {
    note_launches(1);
    k_fill_lut<<<(n_tiles + 255) / 256, 256, 0, s>>>(nb, bstart, n_tiles, lut);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const CamSet *cams_dev, int view, const float4 *qrec, const unsigned long long *gpairs,
                             const int2 *granges, const unsigned long long *ppairs, const int2 *pranges,
                             const int2 *lut, const int *n_blocks, long long max_blocks, const float *pts,
                             float near_plane, float t_stop, bool level_set, float *opacity_out, DevStatus *status,
                             cudaStream_t s) {
    if (max_blocks <= 0) return cudaSuccess;
    note_launches(1);
    k_integrate<<<(unsigned)max_blocks, kQThreads, 0, s>>>(cams_dev, view, qrec, gpairs, granges, ppairs, pranges, lut,
                                                           n_blocks, pts, near_plane, t_stop, level_set, opacity_out,
                                                           status);
    return cudaGetLastError();
}

namespace {
// Bisection along edges for the 0.5 level set: midpoints, then the move of one endpoint.
__global__ void k_midpoints(const float *__restrict__ inside, const float *__restrict__ outside, long long n,
                            float *__restrict__ mid) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3 * n) mid[i] = 0.5f * (inside[i] + outside[i]);
}

__global__ void k_bisect_update(float *__restrict__ inside, float *__restrict__ outside, const float *__restrict__ mid,
                                const float *__restrict__ o_mid, long long n) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float *dst = o_mid[e] > 0.5f ? inside : outside;
    for (int c = 0; c < 3; ++c) dst[3 * e + c] = mid[3 * e + c];
}
}  // namespace

cudaError_t launch_midpoints(const float *inside, const float *outside, long long n, float *mid, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    note_launches(1);
    k_midpoints<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(inside, outside, n, mid);
    return cudaGetLastError();
}

cudaError_t launch_bisect_update(float *inside, float *outside, const float *mid, const float *o_mid, long long n,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    note_launches(1);
    k_bisect_update<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(inside, outside, mid, o_mid, n);
    return cudaGetLastError();
}

}  // namespace sof
