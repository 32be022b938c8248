// Per-(Gaussian, view) preprocessing and tile binning.
//
// k_preprocess builds one 128-byte record per (Gaussian, view) (layout in record.cuh), a
// conservative screen rectangle of the Gaussian's E-ellipsoid silhouette (E from Eq. 3) and a
// lower bound on the peak distance t* of any hit. k_bin_append (one thread per (record, tile of
// its rectangle)) tests the tile against the exact silhouette and the near plane and appends the
// passing (tile, depth key, record) pairs, the key a per-tile lower bound on t* (render) or the
// camera-z of the ellipsoid (query). Bucketed by tile and sorted (tilesort.cu), they give each tile
// a stream of records whose lower bounds never decrease, which the composite kernels merge into
// exact per-pixel t* order.
#include <limits.h>
#include <algorithm>
#include <math.h>

#include "geometry.cuh"
#include "record.cuh"
#include "sof_internal.cuh"

namespace sof {
namespace {


// Writes the record, aux entry and tile rectangle of a visible (Gaussian, view) (layout in
// record.cuh).
__device__ __forceinline__ void emit_record(const SceneDev &sc, const GaussView &G, long long g, long long idx,
                                            int tile, bool query_records, float4 *__restrict__ records,
                                            float4 *__restrict__ aux, int4 *__restrict__ rects) {
    const int px0 = G.px0, px1 = G.px1, py0 = G.py0, py1 = G.py1;  // inclusive pixel bounding box
    float4 *rec = records + idx * kRecF4;
    rec[0] = make_float4(G.ia, G.ja, G.E2 * kPreTest, G.o);
    rec[1] = make_float4(G.c1, G.c2, G.p1, G.q1);
    rec[2] = make_float4(G.q2, dot3(G.og, G.dga), dot3(G.og, G.a), dot3(G.og, G.b));
    rec[3] = make_float4(G.dga.x, G.dga.y, G.dga.z, G.a.x);
    rec[4] = make_float4(G.a.y, G.a.z, G.b.x, G.b.y);
    if (!query_records) {
        // colour from SH along normalize(mu - c); normal = smallest axis facing the camera
        int K = (sc.sh_degree + 1) * (sc.sh_degree + 1);
        F3 dir = (1.f / fmaxf(G.dist, 1e-30f)) * G.w;
        float Y[16];
        sh_eval_basis(sc.sh_degree, dir, Y);
        const float *shp = sc.sh + (size_t)g * K * 3;
        float col[3] = {0.5f, 0.5f, 0.5f};
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) col[ch] = fmaf(Y[k], shp[k * 3 + ch], col[ch]);
        F3 nrm = f3(G.R[0][G.kmin], G.R[1][G.kmin], G.R[2][G.kmin]);
        if (dot3(nrm, G.w) > 0.f) nrm = -1.f * nrm;
        rec[5] = make_float4(G.b.z, fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f));
        rec[6] = make_float4(nrm.x, nrm.y, nrm.z, G.E2);
        rec[7] = make_float4((float)px0, (float)px1, (float)py0, (float)py1);
    } else {
        const float zhi = (float)G.xc[2], zlo = (float)(G.xc[2] - (double)zhi);
        rec[5] = make_float4(G.b.z, 0.f, 0.f, 0.f);
        rec[6] = make_float4(G.delta_x, G.delta_y, zhi, zlo);
        rec[7] = make_float4(G.zmin, G.proj_ok ? 1.f : 0.f, 0.f, 0.f);
    }
    aux[idx] = make_float4(G.t_lo, G.rho2, G.zmin, 1.f);
    rects[idx] = make_int4(px0 / tile, py0 / tile, px1 / tile + 1, py1 / tile + 1);
}

// Render records: two phases per CTA. First every thread runs the culling tests of its (Gaussian,
// view) and the survivors (a few percent in an unbounded scene) are listed in shared memory; then
// the CTA's threads build the survivors' records from that list, densely, so that the FP64 set-up
// of a record (slow on GB300) is not issued for warps that are mostly culled lanes. Query
// records (most of a view's Gaussians survive its culls) take one pass.
__global__ void __launch_bounds__(256) k_preprocess(SceneDev sc, const CamSet *__restrict__ cams,
                                                    float near_plane, bool query_records,
                                                    float4 *__restrict__ records, float4 *__restrict__ aux,
                                                    int4 *__restrict__ rects, DevStatus *status) {
    __shared__ short s_list[256];
    __shared__ int s_n;
    const long long base = (long long)blockIdx.x * blockDim.x;
    const long long n = sc.n;
    const int nv = cams->n_views;
    const int tile = cams->tile;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    bool survives = false, nonfinite = false;
    {
        const long long idx = base + threadIdx.x;
        if (idx < n * nv) {
            const int v = nv == 1 ? 0 : (int)(idx / n);
            const long long g = idx - (long long)v * n;
            GaussView G;
            survives = gauss_view(sc, g, cams->cam[v], near_plane, G, &nonfinite, !query_records);
            if (v != 0) nonfinite = false;
            if (!survives) {
                aux[idx] = make_float4(0.f, -1.f, 0.f, 0.f);
                rects[idx] = make_int4(0, 0, 0, 0);
            } else if (query_records) {
                emit_record(sc, G, g, idx, tile, true, records, aux, rects);
            }
        }
    }
    const unsigned s_mask = __ballot_sync(0xffffffffu, survives);
    const unsigned nf_mask = __ballot_sync(0xffffffffu, nonfinite);
    if (query_records) {
        if (lane == 0) {
            if (s_mask) add_count(status, kCntVisible, (unsigned long long)__popc(s_mask));
            if (nf_mask) atomicAdd(&status->nonfinite, (unsigned long long)__popc(nf_mask));
        }
        return;
    }
    // block-aggregated counters and the survivors' list
    int pos0 = 0;
    if (lane == 0) {
        if (s_mask) pos0 = atomicAdd(&s_n, __popc(s_mask));
        if (nf_mask) atomicAdd(&status->nonfinite, (unsigned long long)__popc(nf_mask));
    }
    pos0 = __shfl_sync(0xffffffffu, pos0, 0);
    if (survives) s_list[pos0 + __popc(s_mask & ((1u << lane) - 1u))] = (short)threadIdx.x;
    __syncthreads();
    const int ns = s_n;
    if (threadIdx.x == 0 && ns) add_count(status, kCntVisible, (unsigned long long)ns);
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        const long long idx = base + s_list[j];
        const int v = nv == 1 ? 0 : (int)(idx / n);
        const long long g = idx - (long long)v * n;
        GaussView G;
        // the same tests pass again: the record's expansion follows
        if (gauss_view(sc, g, cams->cam[v], near_plane, G, nullptr)) {
            emit_record(sc, G, g, idx, tile, false, records, aux, rects);
        } else {
            aux[idx] = make_float4(0.f, -1.f, 0.f, 0.f);
            rects[idx] = make_int4(0, 0, 0, 0);
        }
    }
}

// Test whether the silhouette of a record meets the pixel-centre rectangle of tile (tx, ty).
// In Gaussian space the silhouette is the circular cone |(c1, c2)| / |od| <= rho around o_g;
// pixel positions map to (U, V) = (c1, c2) / od by a projective map, so the tile becomes a convex
// quadrilateral and the test is disc-versus-quadrilateral.
// Also returns a lower bound on t*' = -od/A over the tile (t* in camera-z units of the
// unnormalised ray d' = (u, v, 1), so t* = t*' |d'|). With -od affine and positive on the tile and
// A convex, {t*' >= c} = {-od - c A >= 0} is convex for every c > 0: t*' is quasi-concave there,
// so its minimum over the rectangle is attained at a corner and the bound is exact. Within one
// pixel |d'| is constant, so t*' orders the pixel's hits exactly as the Euclidean t* does.
struct TileTest {
    bool hit;
    float t_lo;      // min over the tile of t*' (0 when -od is not positive on the whole tile)
    float dmax;      // max over the tile of |d'|
};

// Whether the closest point of the edge P -> Q to the origin lies in the disc of squared radius
// rho2, and the cross product P x Q, whose sign says on which side of the edge the origin lies.
__device__ __forceinline__ bool edge_in_disc(float pu, float pv, float qu, float qv, float rho2, float &cr) {
    const float ex = qu - pu, ey = qv - pv;
    cr = ex * (-pv) - ey * (-pu);
    const float ee = ex * ex + ey * ey;
    // any point of the edge gives a valid test; the closest one (up to the approximate division, a
    // second-order change in the distance) gives the tightest
    const float tt = ee > 0.f ? fminf(fmaxf(__fdividef(-(pu * ex + pv * ey), ee), 0.f), 1.f) : 0.f;
    const float qx = pu + tt * ex, qy = pv + tt * ey;
    return qx * qx + qy * qy <= rho2;
}

__device__ __forceinline__ TileTest tile_test(const float4 &r0, const float4 &r1, const float4 &r2,
                                              const float4 &r3, const float4 &r4, const float4 &r5, float rho2,
                                              int px0, int px1, int py0, int py1, float pad,
                                              float near_plane, const DevCam &cam) {
    TileTest res;
    // pixel-centre offsets of the tile's corners; `pad` = 0.5 widens the rectangle to the whole
    // tile area for query points, which lie anywhere in their pixel
    const float x0 = (float)px0 - r0.x - pad, x1 = (float)px1 - r0.x + pad;
    const float y0 = (float)py0 - r0.y - pad, y1 = (float)py1 - r0.y + pad;
    // corners k0 = (x0, y0), k1 = (x1, y0), k2 = (x1, y1), k3 = (x0, y1), visited in that order; each
    // edge k-1 -> k is tested as soon as its second corner is known, the last one k3 -> k0 at the end
    float min_tp = 3.4e38f, max_nod = -3.4e38f;
    bool any_front_bad = false, geo_hit = false, same = true;
    float u_first = 0.f, v_first = 0.f, u_prev = 0.f, v_prev = 0.f, s0 = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float dx = (k == 1 || k == 2) ? x1 : x0, dy = k >= 2 ? y1 : y0;
        const RecEval e = rec_eval(r0, r1, r2, r3, r4, r5, dx, dy);
        const float od = rec_od(r2, e.dx, e.dy);
        if (!(od < 0.f)) any_front_bad = true;
        max_nod = fmaxf(max_nod, -od);
        // U, V only feed the disc test, whose radius carries a relative slack of 1e-4 (kPreTest):
        // an approximate reciprocal (a few ulp) is far inside it
        const float inv = __fdividef(1.f, od);
        const float u = e.c1 * inv, v = e.c2 * inv;
        // the same arithmetic as the per-pixel t*' of the composite kernels
        min_tp = fminf(min_tp, __fmul_rn(-od, rec_rcp(e.A)));
        geo_hit |= u * u + v * v <= rho2;
        if (k == 0) {
            u_first = u;
            v_first = v;
        } else {
            float cr;
            geo_hit |= edge_in_disc(u_prev, v_prev, u, v, rho2, cr);
            // origin inside the quadrilateral: all edge cross products of one sign
            if (k == 1) s0 = cr;
            else same &= cr * s0 >= 0.f;
        }
        u_prev = u;
        v_prev = v;
    }
    {
        float cr;
        geo_hit |= edge_in_disc(u_prev, v_prev, u_first, v_first, rho2, cr);
        same &= cr * s0 >= 0.f;
    }
    // approximate divisions: dmax enters the key, shaved by 2e-5 relative, and the culling bound,
    // padded by 1e-3 relative; a few ulp stay far inside both
    float ua = __fdividef((float)px0 + 0.5f - cam.cx, cam.fx), ub = __fdividef((float)px1 + 0.5f - cam.cx, cam.fx);
    float va = __fdividef((float)py0 + 0.5f - cam.cy, cam.fy), vb = __fdividef((float)py1 + 0.5f - cam.cy, cam.fy);
    float um = fmaxf(fabsf(ua), fabsf(ub)), vm = fmaxf(fabsf(va), fabsf(vb));
    res.dmax = sqrtf(1.f + um * um + vm * vm);  // |d'| is convex: its max is at a corner
    res.t_lo = any_front_bad ? 0.f : fmaxf(min_tp, 0.f);
    // Upper bound on t*' = -od / A over the rectangle: -od is affine (max at a corner) and
    // |d_g| >= |d_g(centre)| - |a| hx - |b| hy. A hit needs t*' |d'| > near, so a tile whose bound
    // stays below near / max|d'| has no hit (a Gaussian behind or around the camera, say).
    if (!(max_nod > 0.f)) {
        res.hit = false;
        return res;
    }
    {
        const float xm = 0.5f * (x0 + x1), ym = 0.5f * (y0 + y1);
        const float hx = 0.5f * (x1 - x0), hy = 0.5f * (y1 - y0);
        const float gx = fmaf(ym, r4.z, fmaf(xm, r3.w, r3.x));
        const float gy = fmaf(ym, r4.w, fmaf(xm, r4.x, r3.y));
        const float gz = fmaf(ym, r5.x, fmaf(xm, r4.y, r3.z));
        const float na = sqrtf(r3.w * r3.w + r4.x * r4.x + r4.y * r4.y);
        const float nb = sqrtf(r4.z * r4.z + r4.w * r4.w + r5.x * r5.x);
        const float lo = sqrtf(gx * gx + gy * gy + gz * gz) - (na * hx + nb * hy);
        if (lo > 0.f && __fdividef(max_nod, lo * lo) * res.dmax * 1.001f < near_plane) {
            res.hit = false;
            return res;
        }
    }
    // a camera inside the ellipsoid, or a corner not in front of it: no silhouette to test
    res.hit = rho2 < 0.f || any_front_bad || geo_hit || same;
    return res;
}

// Upper bound on a record's pairs: the tiles of its rectangle (0 for culled records), and a flag
// for records that have any.
__global__ void k_rect_area(const float4 *__restrict__ aux, const int4 *__restrict__ rects, long long n_rec,
                            int *__restrict__ area, int *__restrict__ flag) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rec) return;
    const int4 rc = rects[i];
    const int a = aux[i].w != 0.f ? (rc.z - rc.x) * (rc.w - rc.y) : 0;
    area[i] = a;
    flag[i] = a > 0 ? 1 : 0;
}

// Compacts the records that have tiles: vis_list[k] = record, vis_area[k] = its tile count.
// A record whose rank reaches vis_cap has no gradient slot: counted in *dropped (the forward
// refuses such a call unless it runs without its host round trip).
__global__ void k_compact_visible(const int *__restrict__ area, const int *__restrict__ flag,
                                  const int *__restrict__ pos, long long n_rec, int *__restrict__ vis_list,
                                  int *__restrict__ vis_area, long long vis_cap,
                                  unsigned long long *__restrict__ dropped) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rec || !flag[i]) return;
    vis_list[pos[i]] = (int)i;
    vis_area[pos[i]] = area[i];
    if (dropped && pos[i] >= vis_cap) atomicAdd(dropped, 1ull);
}

// Render binning in one load-balanced pass: one thread per (record, tile of its rectangle) item,
// items numbered by the exclusive scan vis_off of the compacted records' tile counts (64-bit: a
// call over many views can hold more than 2^31 items). Each CTA finds the records of its 256 items
// (at most 256, each has at least one tile) with one global binary search and a shared-memory
// window. A pair that passes the tile test is appended, at a warp-reserved position, to an unsorted
// list of (global tile, depth key bits, record) and counted in its tile. The depth key is a lower
// bound on t*' of any hit of the record in the tile. With ptile == nullptr the pass only counts the
// pairs that pass (into *cursor), writing nothing else: the sizing pass of a workspace reservation.
constexpr int kAppendThreads = 256;

__global__ void __launch_bounds__(kAppendThreads, 5) k_bin_append(
    const CamSet *__restrict__ cams, long long n_per_view, const float4 *__restrict__ records,
    const float4 *__restrict__ aux, const int4 *__restrict__ rects, const int *__restrict__ vis_list,
    const long long *__restrict__ vis_off, const int *__restrict__ n_vis_dev, const long long *__restrict__ n_items_dev,
    long long max_items, const int *__restrict__ block_first, const int *__restrict__ tile_need, bool query_keys,
    float near_plane, long long cap, unsigned long long *__restrict__ cursor, unsigned *__restrict__ ptile,
    unsigned *__restrict__ pkey, unsigned *__restrict__ prec, int *__restrict__ tile_counts,
    unsigned long long *__restrict__ dropped, unsigned *__restrict__ prank) {
    __shared__ long long s_off[kAppendThreads + 1];
    __shared__ int s_first;
    const int n_vis = *n_vis_dev;
    const int n_views = cams->n_views;
    // items beyond the capacity the grid was sized for are not visited: counted as dropped
    const long long n_items = min(*n_items_dev, max_items);
    if (blockIdx.x == 0 && threadIdx.x == 0 && dropped && *n_items_dev > max_items)
        atomicAdd(dropped, (unsigned long long)(*n_items_dev - max_items));
    // grid-stride over blocks of kAppendThreads items (the grid may be sized for a capacity)
    for (long long item0 = (long long)blockIdx.x * kAppendThreads; item0 < n_items;
         item0 += (long long)gridDim.x * kAppendThreads) {
        __syncthreads();  // the previous block of items is done with the window
        if (threadIdx.x == 0) {
            // last compacted record whose first item is <= item0
            if (block_first) {
                s_first = block_first[item0 / kAppendThreads];
            } else {
                int lo = 0, hi = n_vis - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (vis_off[mid] <= item0) lo = mid;
                    else hi = mid - 1;
                }
                s_first = lo;
            }
        }
        __syncthreads();
        const int first = s_first;
        {
            const int k = first + threadIdx.x;
            s_off[threadIdx.x] = k < n_vis ? vis_off[k] : LLONG_MAX;
            if (threadIdx.x == 0)
                s_off[kAppendThreads] = first + kAppendThreads < n_vis ? vis_off[first + kAppendThreads] : LLONG_MAX;
        }
        __syncthreads();
        const long long item = item0 + threadIdx.x;
        bool ok = false;
        float key_depth = 0.f;
        unsigned gt = 0u, rec = 0u;
        if (item < n_items) {
            // window entry w with s_off[w] <= item < s_off[w + 1]
            int lo = 0, hi = kAppendThreads - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= item) lo = mid;
                else hi = mid - 1;
            }
            rec = (unsigned)vis_list[first + lo];
            const unsigned t = (unsigned)(item - s_off[lo]);
            const float4 ax = aux[rec];
            const int4 rc = rects[rec];
            const unsigned ntx = (unsigned)(rc.z - rc.x);
            // records are [view][Gaussian]: fewer than 2^32 of them
            const DevCam &cam = cams->cam[n_views == 1 ? 0 : (int)(rec / (unsigned)n_per_view)];
            const int tile = cams->tile;
            const float4 *r = records + (size_t)rec * kRecF4;
            const int tx = rc.x + (int)(t % ntx), ty = rc.y + (int)(t / ntx);
            const int px0 = tx * tile, py0 = ty * tile;
            const int px1 = min(px0 + tile, cam.W) - 1, py1 = min(py0 + tile, cam.H) - 1;
            gt = (unsigned)(cam.tile_base + ty * cam.tiles_x + tx);
            // a query bins only into tiles that hold points
            if (!tile_need || tile_need[gt] > 0) {
                // query points lie anywhere in their pixel: the query tests the whole tile area
                const TileTest tt = tile_test(r[0], r[1], r[2], r[3], r[4], r[5], ax.y, px0, px1, py0, py1,
                                              query_keys ? 0.5f : 0.f, near_plane, cam);
                ok = tt.hit;
                // render: every hit has Euclidean t* > max(t_lo_global, near), i.e. t*' > that /
                // max|d'|; query: the exact minimum camera z of the E-ellipsoid. A relative shave
                // keeps FP32 rounding of the per-pixel values from undercutting the bound.
                key_depth = (query_keys ? fmaxf(ax.z, 0.f)
                                        : fmaxf(tt.t_lo, __fdividef(fmaxf(ax.x, near_plane), tt.dmax))) *
                            (1.f - 2e-5f);
            }
        }
        const int lane = threadIdx.x & 31;
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (m == 0u) continue;
        if (!ptile) {
            if (lane == 0) atomicAdd(cursor, (unsigned long long)__popc(m));
            continue;
        }
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(cursor, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (ok) {
            const unsigned long long pos = base + (unsigned long long)__popc(m & ((1u << lane) - 1u));
            if (pos < (unsigned long long)cap) {
                ptile[pos] = gt;
                pkey[pos] = __float_as_uint(key_depth);
                prec[pos] = rec;
                if (prank)
                    prank[pos] = (unsigned)atomicAdd(&tile_counts[gt], 1);
                else
                    atomicAdd(&tile_counts[gt], 1);
            } else if (dropped) {
                atomicAdd(dropped, 1ull);
            }
        }
    }
}

}  // namespace

cudaError_t launch_rect_area(const float4 *aux, const int4 *rects, long long n_rec, int *area, int *flag,
                             cudaStream_t s) {
    if (n_rec == 0) return cudaSuccess;
    note_launches(1);
    k_rect_area<<<(unsigned)((n_rec + 255) / 256), 256, 0, s>>>(aux, rects, n_rec, area, flag);
    return cudaGetLastError();
}

cudaError_t launch_compact_visible(const int *area, const int *flag, const int *pos, long long n_rec, int *vis_list,
                                   int *vis_area, long long vis_cap, unsigned long long *dropped, cudaStream_t s) {
    if (n_rec == 0) return cudaSuccess;
    note_launches(1);
    k_compact_visible<<<(unsigned)((n_rec + 255) / 256), 256, 0, s>>>(area, flag, pos, n_rec, vis_list, vis_area,
                                                                       vis_cap, dropped);
    return cudaGetLastError();
}

cudaError_t launch_bin_append(const CamSet *cams_dev, long long n_per_view, const float4 *records, const float4 *aux,
                              const int4 *rects, const int *vis_list, const long long *vis_off, const int *n_vis_dev,
                              const long long *n_items_dev, long long max_items, bool query_keys, float near_plane,
                              long long cap, unsigned long long *cursor, unsigned *ptile, unsigned *pkey,
                              unsigned *prec, int *tile_counts, unsigned long long *dropped, cudaStream_t s,
                              const int *block_first, const int *tile_need, unsigned *prank) {
    if (max_items <= 0) return cudaSuccess;
    note_launches(1);
    const long long blocks = std::min<long long>((max_items + kAppendThreads - 1) / kAppendThreads, (long long)device_sm_count() * 64);
    k_bin_append<<<(unsigned)blocks, kAppendThreads, 0, s>>>(
        cams_dev, n_per_view, records, aux, rects, vis_list, vis_off, n_vis_dev, n_items_dev, max_items, block_first,
        tile_need, query_keys, near_plane, cap, cursor, ptile, pkey, prec, tile_counts, dropped, prank);
    return cudaGetLastError();
}

namespace {
// block_first[b] = the compacted record holding item b * kAppendThreads: each record writes the
// blocks whose first item it holds.
__global__ void k_block_first(const long long *__restrict__ vis_off, const int *__restrict__ n_vis_dev,
                              const long long *__restrict__ n_items_dev, long long max_items,
                              int *__restrict__ block_first) {
    const int n = *n_vis_dev;
    const long long n_items = min(*n_items_dev, max_items);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const long long lo = vis_off[k], hi = min(k + 1 < n ? (long long)vis_off[k + 1] : n_items, n_items);
        for (long long b = (lo + kAppendThreads - 1) / kAppendThreads; b * kAppendThreads < hi; ++b)
            block_first[b] = (int)k;
    }
}
}  // namespace

cudaError_t launch_block_first(const long long *vis_off, const int *n_vis_dev, const long long *n_items_dev,
                               long long max_vis, long long max_items, int *block_first, cudaStream_t s) {
    if (max_vis <= 0 || max_items <= 0) return cudaSuccess;
    note_launches(1);
    const unsigned blocks = (unsigned)std::min<long long>((max_vis + 255) / 256, (long long)device_sm_count() * 8);
    k_block_first<<<blocks, 256, 0, s>>>(vis_off, n_vis_dev, n_items_dev, max_items, block_first);
    return cudaGetLastError();
}

cudaError_t launch_preprocess(const SceneDev &sc, const CamSet *cams_dev, const CamSet &cams_host,
                              float near_plane, bool query_records, float4 *records, float4 *aux,
                              int4 *rects, DevStatus *status, cudaStream_t s) {
    long long total = sc.n * (long long)cams_host.n_views;
    if (total == 0) return cudaSuccess;
    int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    note_launches(1);
    k_preprocess<<<(unsigned)blocks, threads, 0, s>>>(sc, cams_dev, near_plane, query_records, records, aux,
                                                       rects, status);
    return cudaGetLastError();
}

}  // namespace sof
