// Opacity field at 3D points, min over views (Eqs. 11-12, App. A.2; Sec. 3.4 "Ray/Tile
// Scheduling", "Early Stopping").
//
// Per view: the Gaussians are bucketed by screen tile and sorted by z_min within each tile (one
// word z_min bits << 32 | record), z_min the exact minimum camera z of the E-ellipsoid; the visible
// points are bucketed by tile and grouped by camera z (z bits << 32 | point, ordered by the top 16
// bits of z), so that each CTA takes up to 256 points of one tile at similar depths (a block -> tile
// table, as in the paper's scheduling), two per thread. Each point is evaluated
// against the tile's Gaussians in z_min order and stops at the first with z_min > z(point): no
// later one can reach alpha >= 1/255 at t_eval <= t. O_N = 1 - prod(1 - alpha) needs no order
// (App. A.2). A view's running value only grows, so a point's walk also stops once it reaches the
// point's current minimum over the views already done (exact pruning; the min cannot change).
#include <math.h>

#include "record.cuh"
#include "sof_internal.cuh"

namespace sof {
namespace {

constexpr int kQThreads = 256;  // points per block of the block -> tile table
constexpr int kQChunk = 64;

struct PointProj {
    bool vis;
    float Xh, Xl, Yh, Yl, zh, zl, dn;
    int px, py;
};

// Double-float arithmetic: a value is hi + lo, two floats with |lo| <= ulp(hi) / 2, carried on the
// FP32 pipe (FP64 runs at a small fraction of the FP32 rate on GB300). The error-free
// transformations are Knuth's TwoSum and the FMA form of Dekker's TwoProduct; the compound
// operations are the classic double-single ones, accurate to about 2^-44 relative. The explicit
// round-to-nearest intrinsics keep the compiler from contracting or reordering them.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF quick_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    const DF t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    DF p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    DF p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return quick_two_sum(p.hi, p.lo);
}
// 1 / z: a float reciprocal refined by one Newton-Raphson step r + r (1 - z r), the residual
// 1 - z r taken in double-float
__device__ __forceinline__ DF df_recip(DF z) {
    const float r = __frcp_rn(z.hi);
    const DF zr = df_mul_f(z, r);
    const DF e = df_add({1.f, 0.f}, {-zr.hi, -zr.lo});
    return df_add({r, 0.f}, two_prod(r, e.hi));
}
// a < b for double-floats (normalised, so the hi parts decide unless equal)
__device__ __forceinline__ bool df_lt(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

// Camera-space position and projection of a point in double-float: FP32 products are exact as
// TwoProducts, so the camera transform carries no cancellation error; the pixel position and the
// depth come out as hi + lo floats.
__device__ __forceinline__ PointProj project_point(const DevCam &cam, const float *pts, long long i, float near_plane) {
    PointProj r;
    const float x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    DF c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        DF a = two_prod(cam.Rf[3 * k], x);
        a = df_add(a, two_prod(cam.Rf[3 * k + 1], y));
        a = df_add(a, two_prod(cam.Rf[3 * k + 2], z));
        c[k] = df_add(a, {cam.tf[k], 0.f});
    }
    r.vis = false;
    r.px = r.py = 0;
    r.Xh = r.Xl = r.Yh = r.Yl = r.zh = r.zl = r.dn = 0.f;
    if (!df_lt({near_plane, 0.f}, c[2])) return r;
    const DF iz = df_recip(c[2]);
    const DF u = df_mul(c[0], iz), v = df_mul(c[1], iz);
    const DF X = df_add(df_mul_f(u, cam.fx), {cam.cx, 0.f}), Y = df_add(df_mul_f(v, cam.fy), {cam.cy, 0.f});
    const DF zero = {0.f, 0.f};
    if (df_lt(X, zero) || !df_lt(X, {(float)cam.W, 0.f}) || df_lt(Y, zero) || !df_lt(Y, {(float)cam.H, 0.f})) return r;
    r.vis = true;
    r.Xh = X.hi; r.Xl = X.lo;
    r.Yh = Y.hi; r.Yl = Y.lo;
    r.zh = c[2].hi; r.zl = c[2].lo;
    r.dn = sqrtf(1.f + u.hi * u.hi + v.hi * v.hi);  // |d'|, an FP32 value
    // pixel = floor(X): hi rounded down, less one where hi is an integer and lo < 0
    const float fx = floorf(X.hi), fy = floorf(Y.hi);
    r.px = min((int)fx - (fx == X.hi && X.lo < 0.f ? 1 : 0), cam.W - 1);
    r.py = min((int)fy - (fy == Y.hi && Y.lo < 0.f ? 1 : 0), cam.H - 1);
    return r;
}

// Projects every point into the view; a visible one is counted in seen[], counted in its tile and
// appended, at a warp-reserved position, to an unsorted list (tile, z bits, point), with its rank
// among its tile's points.
__global__ void __launch_bounds__(256) k_point_append(const CamSet *__restrict__ cams, int view,
                                                      const float *__restrict__ pts, long long n_points,
                                                      float near_plane, int *__restrict__ seen,
                                                      unsigned long long *__restrict__ cursor,
                                                      unsigned *__restrict__ ptile,
                                                      unsigned *__restrict__ pkey, unsigned *__restrict__ pidx,
                                                      unsigned *__restrict__ prank, int *__restrict__ tile_counts) {
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
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (vis) {
        // at most one entry per point: positions stay below n_points
        const unsigned long long pos = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
        ptile[pos] = gt;
        pkey[pos] = key;
        pidx[pos] = (unsigned)i;
    }
    // the point's rank in its tile: one atomic per tile among the warp's lanes (neighbouring
    // points mostly share a tile), so that the bucketing places each point without an atomic
    const unsigned peers = __match_any_sync(0xffffffffu, vis ? gt : 0xFFFFFFFFu) & m;
    int rank0 = 0;
    if (vis && (peers & ((1u << lane) - 1u)) == 0u) rank0 = atomicAdd(&tile_counts[gt], __popc(peers));
    rank0 = __shfl_sync(0xffffffffu, rank0, vis ? __ffs(peers) - 1 : lane);
    if (vis) {
        const unsigned long long pos = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
        prank[pos] = (unsigned)(rank0 + __popc(peers & ((1u << lane) - 1u)));
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

// One point's walk through its tile's list.
struct PointWalk {
    long long pi;
    PointProj pp;
    float P, stop_at;
    bool done;
};

// Sets up point q of the block (q >= np: nothing to do).
__device__ __forceinline__ void walk_init(PointWalk &w, const DevCam &cam, const unsigned long long *ppairs,
                                          const float *pts, const float *opacity_out, int p0, int q, int np,
                                          float near_plane, float t_stop, bool level_set) {
    w.done = q >= np;
    w.pi = 0;
    w.pp.vis = false;
    w.P = 1.f;
    w.stop_at = 0.f;
    if (w.done) return;
    w.pi = (unsigned)ppairs[p0 + q];
    w.pp = project_point(cam, pts, w.pi, near_plane);
    const float cur = opacity_out[w.pi];  // running min over the views done so far
    // stop once 1 - P >= cur (this view cannot lower the min any more), P < t_stop, or P <= 2^-25:
    // from there on 1 - P rounds to 1.0f whatever is multiplied in, so stopping leaves the FP32
    // result unchanged
    w.stop_at = fmaxf(fmaxf(1.f - cur, t_stop), 0x1p-25f);
    w.done = !w.pp.vis || cur <= 0.f;
    if (level_set) {
        // only O > 0.5 matters: this view is done once 1 - P > 0.5 (P below 0.5, the largest float
        // under 0.5 being 0.5 - 2^-25), and a point some view left at O <= 0.5 is out
        w.stop_at = fmaxf(w.stop_at, 0.5f - 0x1p-25f);
        w.done = w.done || cur <= 0.5f;
    }
}

// One (point, Gaussian) evaluation, the record's first six float4 at hand and its seventh (the
// query fields) in shared memory.
__device__ __forceinline__ void walk_step(PointWalk &w, const float4 &r0, const float4 &r1, const float4 &r2,
                                          const float4 &r3, const float4 &r4, const float4 &r5,
                                          const float4 *r6p, bool proj, float near_plane, unsigned &n_tests,
                                          unsigned &n_inc) {
    const PointProj &pp = w.pp;
    // offset from the anchor pixel centre (ia + 0.5, ja + 0.5), cancellation-free
    const float dx = (pp.Xh - (r0.x + 0.5f)) + pp.Xl;
    const float dy = (pp.Yh - (r0.y + 0.5f)) + pp.Yl;
    const RecEval e = rec_eval(r0, r1, r2, r3, r4, r5, dx, dy);
    ++n_tests;
    if (!(e.N <= __fmul_rn(r0.z, e.A))) return;  // the line misses the E-ellipsoid
    const float rA = rec_rcp(e.A);
    const float m = __fmul_rn(e.N, rA);
    float tstar, behind;  // peak t*' (camera-z units) and z(point) - t*'
    if (proj) {
        const float4 r6 = *r6p;
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
        w.P *= (1.f - a);
        if (w.P <= w.stop_at) w.done = true;
    }
}

// Each thread walks PPT points of the block (consecutive in depth order), so that every record
// read from shared memory serves all of them: two where the blocks are full (fewer shared-memory
// loads per evaluation), one where tiles hold few points (more threads to hide the latency).
template <int PPT>
__global__ void __launch_bounds__(kQThreads / PPT) k_integrate(const CamSet *__restrict__ cams, int view,
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
    constexpr int CTA = kQThreads / PPT;
    PointWalk w[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k)
        walk_init(w[k], cam, ppairs, pts, opacity_out, p0, PPT * tid + k, np, near_plane, t_stop, level_set);
    auto all_done = [&]() {
        bool d = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) d = d && w[k].done;
        return d;
    };
    unsigned n_tests = 0, n_inc = 0;
    for (int base = gr.x; base < gr.y; base += kQChunk) {
        const int n = min(kQChunk, gr.y - base);
        __syncthreads();
        for (int i = tid; i < n * 7; i += CTA) {
            const int j = i / 7, f = i - j * 7;
            srec[f][j] = qrec[(size_t)(unsigned)gpairs[base + j] * kRecF4 + f];
        }
        for (int i = tid; i < n; i += CTA) {
            const unsigned long long g = gpairs[base + i];
            szmin[i] = __uint_as_float((unsigned)(g >> 32));
            sproj[i] = qrec[(size_t)(unsigned)g * kRecF4 + 7].y;
        }
        __syncthreads();
        for (int j = 0; j < n && !all_done(); ++j) {
            // z_min order: no later Gaussian can contribute to a point in front of this one's z_min
            const float zmin = szmin[j];
#pragma unroll
            for (int k = 0; k < PPT; ++k) w[k].done = w[k].done || zmin > w[k].pp.zh;
            if (all_done()) break;
            const float4 r0 = srec[0][j], r1 = srec[1][j], r2 = srec[2][j], r3 = srec[3][j], r4 = srec[4][j],
                         r5 = srec[5][j];
            const bool proj = sproj[j] != 0.f;
#pragma unroll
            for (int k = 0; k < PPT; ++k)
                if (!w[k].done)
                    walk_step(w[k], r0, r1, r2, r3, r4, r5, &srec[6][j], proj, near_plane, n_tests, n_inc);
        }
        if (__syncthreads_and(all_done())) break;
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (PPT * tid + k < np && w[k].pp.vis) {
            const float O = 1.f - w[k].P;
            if (O < opacity_out[w[k].pi]) atomicMin(reinterpret_cast<int *>(opacity_out + w[k].pi), __float_as_int(O));
        }
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
                               float near_plane, int *seen, unsigned long long *cursor, unsigned *ptile,
                               unsigned *pkey, unsigned *pidx, unsigned *prank, int *tile_counts, cudaStream_t s) {
    if (n_points <= 0) return cudaSuccess;
    note_launches(1);
    k_point_append<<<(unsigned)((n_points + 255) / 256), 256, 0, s>>>(cams_dev, view, pts, n_points, near_plane, seen,
                                                                       cursor, ptile, pkey, pidx, prank, tile_counts);
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
                             long long points_per_tile, cudaStream_t s) {
    if (max_blocks <= 0) return cudaSuccess;
    note_launches(1);
    if (points_per_tile >= 1024)
        k_integrate<2><<<(unsigned)max_blocks, kQThreads / 2, 0, s>>>(cams_dev, view, qrec, gpairs, granges, ppairs,
                                                                      pranges, lut, n_blocks, pts, near_plane, t_stop,
                                                                      level_set, opacity_out, status);
    else
        k_integrate<1><<<(unsigned)max_blocks, kQThreads, 0, s>>>(cams_dev, view, qrec, gpairs, granges, ppairs,
                                                                  pranges, lut, n_blocks, pts, near_plane, t_stop,
                                                                  level_set, opacity_out, status);
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
