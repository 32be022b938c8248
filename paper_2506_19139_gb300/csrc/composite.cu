// Exact-order front-to-back compositing per pixel (forward and backward).
//
// One CTA per screen tile, one thread per pixel. The tile's records arrive sorted by a lower
// bound on the peak t*' (camera-z units) of any of their hits inside the tile (k_bin). Records are
// staged into shared memory in chunks; each pixel tests each record with the anchored closed form
// (m = |cross|^2/A <= E^2 pre-test, then alpha = min(0.99, o exp(-m/2)) >= 1/255 and t* > near,
// Sec. 3.1 Eqs. 9-10), and keeps its hits in a small per-pixel buffer sorted by (t*', record). A
// buffered hit is composited once its t*' is below the key of every record not yet tested, which
// makes the composite order exactly the ascending t* order of Sec. 3.1 ("StopThePop" per-ray
// sorting; |d'| is constant within a pixel, so t*' and t* order alike). Transmittance
// T' = T (1 - alpha) stops the pixel before the hit that would drop T below t_stop. The 0.5
// crossing gives the exact depth of Sec. 3.2 / App. A.3.
//
// A pixel whose buffer would overflow is abandoned by the main kernel, marked, and recomputed
// exactly by k_composite_fallback (one warp per pixel, selection of the next hit in order), so the
// result is exact for any buffer size.
//
// The backward replays the identical decisions front to back (the same evaluation code runs),
// using the forward's final sums for the contributions of later hits (App. C.1 uses the same
// front-to-back pattern), and accumulates per-record gradients with float4 atomics.
#include <math.h>

#include "record.cuh"
#include "sof_internal.cuh"

namespace sof {
namespace {

constexpr float kInf = 3.402823466e38f;

struct PixelGrad {
    float gC[3], gD, gE, gMed, gN[3], gO;
    float Cf[3], Df, Nf[3], Tf;
    float Cacc[3], Dacc, Nacc[3];
};

// Per-pixel compositing state shared by the main kernel and the fallback.
template <bool BWD>
struct Pixel {
    float fpx, fpy, dnorm;
    long long pix, cbase;
    int HW;
    float T;
    float C[3], D, Nn[3];
    int cnt;
    bool crossed, done;
    unsigned r_cross;
    float T_cross, t_cross;
    PixelGrad pg;

    __device__ __forceinline__ void init(const CompositeParams &p, const DevCam &cam, int px, int py) {
        fpx = (float)px;
        fpy = (float)py;
        const float uu = ((float)px + 0.5f - cam.cx) / cam.fx, vv = ((float)py + 0.5f - cam.cy) / cam.fy;
        dnorm = sqrtf(1.f + uu * uu + vv * vv);
        HW = cam.W * cam.H;
        pix = cam.pix_base + (long long)py * cam.W + px;
        cbase = 3 * cam.pix_base + (long long)py * cam.W + px;
        T = 1.f;
        for (int c = 0; c < 3; ++c) C[c] = Nn[c] = 0.f;
        D = 0.f;
        cnt = 0;
        crossed = done = false;
        r_cross = 0;
        T_cross = t_cross = 0.f;
        if (BWD) {
            for (int c = 0; c < 3; ++c) {
                pg.gC[c] = p.d_color ? p.d_color[cbase + (long long)c * HW] : 0.f;
                pg.gN[c] = p.d_normal ? p.d_normal[cbase + (long long)c * HW] : 0.f;
                pg.Nf[c] = p.normal[cbase + (long long)c * HW];
                pg.Cacc[c] = 0.f;
                pg.Nacc[c] = 0.f;
            }
            pg.gD = p.d_depth ? p.d_depth[pix] : 0.f;
            pg.gE = p.d_exact ? p.d_exact[pix] : 0.f;
            pg.gMed = p.d_median ? p.d_median[pix] : 0.f;
            pg.gO = p.d_opacity ? p.d_opacity[pix] : 0.f;
            pg.Tf = 1.f - p.opacity[pix];
            for (int c = 0; c < 3; ++c) pg.Cf[c] = p.color[cbase + (long long)c * HW] - pg.Tf * p.bg[c];
            pg.Df = p.depth[pix];
            pg.Dacc = 0.f;
        }
    }

    // Composite the next hit in order (t*' = tp); `emit` selects the thread that issues the
    // gradient atomics (the fallback runs a pixel on a whole warp).
    __device__ __forceinline__ void composite(const CompositeParams &p, float tp, float a, unsigned r, bool emit) {
        const float t = __fmul_rn(tp, dnorm);  // Euclidean t*
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
        if (Tn < p.t_stop) {
            done = true;
            return;
        }
        const float w = __fmul_rn(a, T);
        const float4 *rp = p.records + (size_t)r * kRecF4;
        const float4 q5 = rp[5], q6 = rp[6];
        const float rgb[3] = {q5.y, q5.z, q5.w}, nr[3] = {q6.x, q6.y, q6.z};
        const bool is_cross = !crossed && T > 0.5f && Tn <= 0.5f;
        if (!BWD) {
            for (int c = 0; c < 3; ++c) {
                C[c] = fmaf(w, rgb[c], C[c]);
                Nn[c] = fmaf(w, nr[c], Nn[c]);
            }
            D = fmaf(w, t, D);
            if (is_cross) {
                crossed = true;
                r_cross = r;
                T_cross = T;
                t_cross = t;
            }
        } else {
            if (is_cross) crossed = true;
            for (int c = 0; c < 3; ++c) {
                pg.Cacc[c] = fmaf(w, rgb[c], pg.Cacc[c]);
                pg.Nacc[c] = fmaf(w, nr[c], pg.Nacc[c]);
            }
            pg.Dacc = fmaf(w, t, pg.Dacc);
            const float dLdt = w * pg.gD + (is_cross ? pg.gE + pg.gMed : 0.f);
            const float inv = 1.f / (1.f - a);
            const float front = pg.gC[0] * rgb[0] + pg.gC[1] * rgb[1] + pg.gC[2] * rgb[2] + pg.gD * t +
                                pg.gN[0] * nr[0] + pg.gN[1] * nr[1] + pg.gN[2] * nr[2];
            const float behind = pg.gC[0] * (pg.Cf[0] - pg.Cacc[0]) + pg.gC[1] * (pg.Cf[1] - pg.Cacc[1]) +
                                 pg.gC[2] * (pg.Cf[2] - pg.Cacc[2]) + pg.gD * (pg.Df - pg.Dacc) +
                                 pg.gN[0] * (pg.Nf[0] - pg.Nacc[0]) + pg.gN[1] * (pg.Nf[1] - pg.Nacc[1]) +
                                 pg.gN[2] * (pg.Nf[2] - pg.Nacc[2]);
            const float bgterm = pg.gO - (pg.gC[0] * p.bg[0] + pg.gC[1] * p.bg[1] + pg.gC[2] * p.bg[2]);
            const float dLda = T * front - behind * inv + bgterm * pg.Tf * inv;
            // re-evaluate the record at this pixel (same arithmetic as the test)
            const float4 q0 = rp[0];
            const RecEval q = rec_eval(q0, rp[1], rp[2], rp[3], rp[4], q5, fpx - q0.x, fpy - q0.y);
            const float c1 = q.c1, c2 = q.c2;
            const float rA = __frcp_rn(q.A);
            const float m = __fmul_rn(q.N, rA);
            const float G = __expf(-0.5f * m);
            const bool clamped = !(__fmul_rn(q0.w, G) < kAlphaMax);
            const float dLdm = clamped ? 0.f : dLda * (-0.5f * a);
            const float dLdo = clamped ? 0.f : dLda * G;
            const float gNq = dLdm * rA;
            const float gA = -(dLdm * m + dLdt * t) * rA;
            const float god = -dLdt * dnorm * rA;
            const float gc1 = 2.f * gNq * c1, gc2 = 2.f * gNq * c2;
            const float dx = q.dx, dy = q.dy;
            if (emit) {
                float4 *gp = p.rgrad + (size_t)r * kGradF4;
                atomicAdd(gp + 0, make_float4(gc1, gc2, gc1 * dx, gc2 * dx));
                atomicAdd(gp + 1, make_float4(gc1 * dy, gc2 * dy, gA, gA * dx));
                atomicAdd(gp + 2, make_float4(gA * dy, gA * dx * dx, gA * dx * dy, gA * dy * dy));
                atomicAdd(gp + 3, make_float4(god, god * dx, god * dy, dLdo));
                atomicAdd(gp + 4, make_float4(w * pg.gC[0], w * pg.gC[1], w * pg.gC[2], w * pg.gN[0]));
                atomicAdd(gp + 5, make_float4(w * pg.gN[1], w * pg.gN[2], 0.f, 0.f));
            }
        }
        T = Tn;
        ++cnt;
    }

    __device__ __forceinline__ void write_outputs(const CompositeParams &p) {
        for (int c = 0; c < 3; ++c) {
            p.color[cbase + (long long)c * HW] = C[c] + T * p.bg[c];
            p.normal[cbase + (long long)c * HW] = Nn[c];
        }
        p.depth[pix] = D;
        p.opacity[pix] = 1.f - T;
        p.n_contrib[pix] = cnt;
        float ex = 0.f, med = 0.f;
        if (crossed) {
            // exact depth: T_k (1 - o_k G(t)) = 0.5 on the camera side of t*_k (App. A.3)
            const float4 *rp = p.records + (size_t)r_cross * kRecF4;
            const float4 q0 = rp[0];
            const RecEval q = rec_eval(q0, rp[1], rp[2], rp[3], rp[4], rp[5], fpx - q0.x, fpy - q0.y);
            const float m = q.N / q.A;
            const float g = (T_cross - 0.5f) / (T_cross * rp[0].w);
            const float x = -2.f * logf(g) - m;
            const float delta = sqrtf(fmaxf(x, 0.f) / q.A);
            ex = t_cross - delta * dnorm;
            med = t_cross;
        }
        p.exact_depth[pix] = ex;
        if (p.median_depth) p.median_depth[pix] = med;
    }
};

__device__ __forceinline__ int view_of_tile(const CamSet *cs, int gtile) {
    int v = 0;
    while (v + 1 < cs->n_views && cs->cam[v + 1].tile_base <= gtile) ++v;
    return v;
}

template <int TILE, int CHUNK, int K, bool BWD>
__global__ void __launch_bounds__(TILE *TILE) k_composite(CompositeParams p) {
    constexpr int NT = TILE * TILE;
    extern __shared__ float4 smem[];
    float4 *srec = smem;                                              // [kRecStage][CHUNK]
    float *pend_t = reinterpret_cast<float *>(srec + kRecStage * CHUNK);  // [K][NT]
    float *pend_a = pend_t + K * NT;                                  // [K][NT]
    unsigned *pend_r = reinterpret_cast<unsigned *>(pend_a + K * NT); // [K][NT]
    unsigned *sidx = pend_r + K * NT;                                 // [CHUNK]
    float *stlo = reinterpret_cast<float *>(sidx + CHUNK);            // [CHUNK]

    const int tid = threadIdx.x;
    const int gtile = blockIdx.x;
    const DevCam &cam = p.cams->cam[view_of_tile(p.cams, gtile)];
    const int lt = gtile - cam.tile_base;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    const int px = tx * TILE + tid % TILE, py = ty * TILE + tid / TILE;
    const bool inside = px < cam.W && py < cam.H;
    const int2 range = p.ranges[gtile];

    Pixel<BWD> st;
    st.init(p, cam, inside ? px : 0, inside ? py : 0);
    st.done = !inside;
    bool ovf = false;
    if (BWD && inside && p.ovf_mask[st.pix]) st.done = true;  // recomputed by the fallback

    // pending ring [head, head + pcount) sorted by (t*', record)
    int head = 0, pcount = 0;
    float head_t = kInf, last_t = -kInf;
    bool inexact = false;
    unsigned n_tests = 0, n_hits = 0, n_below = 0;

    auto pop = [&]() {
        const int sl = head * NT + tid;
        const float t = pend_t[sl], a = pend_a[sl];
        const unsigned r = pend_r[sl];
        head = (head + 1) & (K - 1);
        --pcount;
        head_t = pcount > 0 ? pend_t[head * NT + tid] : kInf;
        last_t = t;
        st.composite(p, t, a, r, true);
    };

    auto insert = [&](float t, float a, unsigned r) {
        if (t < last_t) inexact = true;  // arrives behind a hit already composited
        if (pcount == K) {
            // the buffer is full: leave this pixel to the exact fallback
            ovf = true;
            st.done = true;
            return;
        }
        int pos = pcount;
        while (pos > 0) {
            const int sl = ((head + pos - 1) & (K - 1)) * NT + tid;
            const float tt = pend_t[sl];
            if (tt < t || (tt == t && pend_r[sl] < r)) break;
            const int dl = ((head + pos) & (K - 1)) * NT + tid;
            pend_t[dl] = tt;
            pend_a[dl] = pend_a[sl];
            pend_r[dl] = pend_r[sl];
            --pos;
        }
        const int dl = ((head + pos) & (K - 1)) * NT + tid;
        pend_t[dl] = t;
        pend_a[dl] = a;
        pend_r[dl] = r;
        ++pcount;
        if (pos == 0) head_t = t;
    };

    for (int base = range.x; base < range.y; base += CHUNK) {
        const int n = min(CHUNK, range.y - base);
        __syncthreads();
        for (int i = tid; i < n; i += NT) {
            sidx[i] = p.vals[base + i];
            stlo[i] = __uint_as_float((unsigned)(p.keys[base + i] & 0xFFFFFFFFull));
        }
        __syncthreads();
        for (int i = tid; i < n * kRecStage; i += NT) {
            const int j = i / kRecStage, f = i - j * kRecStage;
            srec[f * CHUNK + j] = p.records[(size_t)sidx[j] * kRecF4 + f];
        }
        const float tlo_after =
            (base + n < range.y) ? __uint_as_float((unsigned)(p.keys[base + n] & 0xFFFFFFFFull)) : kInf;
        if (!BWD && tid == 0) {
            // the merge needs non-decreasing keys within the tile's stream
            bool sorted = true;
            for (int i = 1; i < n; ++i) sorted &= !(stlo[i] < stlo[i - 1]);
            sorted &= !(tlo_after < stlo[n - 1]);
            if (!sorted) atomicAdd(&p.status->n_unsorted, 1ull);
        }
        __syncthreads();
        if (!st.done) {
            int j = 0;
            for (; j < n; ++j) {
                const float4 r0 = srec[j], r1 = srec[CHUNK + j], r2 = srec[2 * CHUNK + j], r3 = srec[3 * CHUNK + j];
                const float4 r4 = srec[4 * CHUNK + j], r5 = srec[5 * CHUNK + j];
                const RecEval q = rec_eval(r0, r1, r2, r3, r4, r5, st.fpx - r0.x, st.fpy - r0.y);
                if (q.N <= __fmul_rn(r0.z, q.A)) {
                    float tp, a;
                    if (rec_hit(q, r0, r2, st.dnorm, p.near_plane, tp, a)) {
                        ++n_hits;
                        n_below += (tp < stlo[j]);
                        insert(tp, a, sidx[j]);
                        if (st.done) break;
                    }
                }
                const float tn = (j + 1 < n) ? stlo[j + 1] : tlo_after;
                while (pcount > 0 && head_t < tn) {
                    pop();
                    if (st.done) break;
                }
                if (st.done) break;
            }
            n_tests += (unsigned)min(j + 1, n);
        }
        if (__syncthreads_and(st.done)) break;
    }
    while (!st.done && pcount > 0) pop();

    if (!BWD && inside) {
        p.ovf_mask[st.pix] = ovf ? 1 : 0;
        if (ovf) {
            atomicAdd(&p.status->n_forced, 1ull);
            const int e = atomicAdd(p.ovf_count, 1);
            p.ovf_list[e] = ((unsigned)gtile << 8) | (unsigned)tid;
        } else {
            st.write_outputs(p);
        }
    }
    if (inexact) atomicAdd(&p.status->inexact_pixels, 1ull);
    if (!BWD) {
        // work counters (one atomic per warp)
        unsigned long long a = n_tests, b = n_hits, c = ovf ? 0u : (unsigned)st.cnt, e = n_below;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
        }
        if ((tid & 31) == 0) {
            atomicAdd(&p.status->n_tests, a);
            atomicAdd(&p.status->n_hits, b);
            atomicAdd(&p.status->n_composited, c);
            if (e) atomicAdd(&p.status->n_below_key, e);
        }
    }
}

// Exact fallback for pixels whose pending buffer overflowed: one warp per pixel selects the next
// hit in (t*', record) order among the tile's records, scanning the key-sorted stream only up to
// the first key above the best candidate so far (no later record can have an earlier hit).
template <int TILE, bool BWD>
__global__ void __launch_bounds__(256) k_composite_fallback(CompositeParams p) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int count = *p.ovf_count;
    for (int e = warp; e < count; e += n_warps) {
        const unsigned code = p.ovf_list[e];
        const int gtile = (int)(code >> 8), tid = (int)(code & 255u);
        const DevCam &cam = p.cams->cam[view_of_tile(p.cams, gtile)];
        const int lt = gtile - cam.tile_base;
        const int px = (lt % cam.tiles_x) * TILE + tid % TILE, py = (lt / cam.tiles_x) * TILE + tid / TILE;
        const int2 range = p.ranges[gtile];
        Pixel<BWD> st;
        st.init(p, cam, px, py);
        unsigned long long last = 0ull;  // (t*' bits << 32 | record) of the last composited hit
        unsigned n_fb = 0;
        while (true) {
            unsigned long long best = ~0ull;
            for (int base = range.x; base < range.y; base += 32) {
                const float kb = __uint_as_float((unsigned)(p.keys[base] & 0xFFFFFFFFull));
                if (best != ~0ull && kb > __uint_as_float((unsigned)(best >> 32))) break;
                const int j = base + lane;
                unsigned long long cand = ~0ull;
                if (j < range.y) {
                    const unsigned r = p.vals[j];
                    const float4 *rp = p.records + (size_t)r * kRecF4;
                    const float4 r0 = rp[0], r2 = rp[2];
                    const RecEval q = rec_eval(r0, rp[1], r2, rp[3], rp[4], rp[5], st.fpx - r0.x, st.fpy - r0.y);
                    float tp, a;
                    if (q.N <= __fmul_rn(r0.z, q.A) && rec_hit(q, r0, r2, st.dnorm, p.near_plane, tp, a)) {
                        const unsigned long long pk = ((unsigned long long)__float_as_uint(tp) << 32) | r;
                        if (pk > last) cand = pk;
                    }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long other = __shfl_xor_sync(0xffffffffu, cand, o);
                    cand = other < cand ? other : cand;
                }
                best = cand < best ? cand : best;
            }
            if (best == ~0ull) break;
            const unsigned r = (unsigned)(best & 0xFFFFFFFFull);
            const float4 *rp = p.records + (size_t)r * kRecF4;
            const float4 r0 = rp[0], r2 = rp[2];
            const RecEval q = rec_eval(r0, rp[1], r2, rp[3], rp[4], rp[5], st.fpx - r0.x, st.fpy - r0.y);
            float tp, a;
            rec_hit(q, r0, r2, st.dnorm, p.near_plane, tp, a);
            st.composite(p, tp, a, r, lane == 0);
            if (st.done) break;
            last = best;
            ++n_fb;
        }
        if (!BWD && lane == 0) {
            st.write_outputs(p);
            atomicAdd(&p.status->n_composited, (unsigned long long)st.cnt);
        }
        (void)n_fb;
    }
}

template <int CHUNK, int K>
size_t smem_bytes(int nt) {
    return (size_t)kRecStage * CHUNK * sizeof(float4) + (size_t)K * nt * 12 + (size_t)CHUNK * 8;
}

template <int CHUNK, int K, bool BWD>
cudaError_t launch_t(const CompositeParams &p, int total_tiles, cudaStream_t s) {
    constexpr int TILE = 16;
    const size_t sm = smem_bytes<CHUNK, K>(TILE * TILE);
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_composite<TILE, CHUNK, K, BWD>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    note_launches(1);
    k_composite<TILE, CHUNK, K, BWD><<<total_tiles, TILE * TILE, sm, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the fallback reads the overflow count on the device; 8 warps per SM-sized block set
    note_launches(1);
    k_composite_fallback<TILE, BWD><<<152 * 4, 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <bool BWD>
cudaError_t dispatch(const CompositeParams &p, int total_tiles, int tile, int chunk, int k, cudaStream_t s) {
    if (total_tiles <= 0) return cudaSuccess;
    if (tile != 16) return cudaErrorInvalidValue;
#define SOF_CASE(CH, KK) \
    if (chunk == CH && k == KK) return launch_t<CH, KK, BWD>(p, total_tiles, s);
    SOF_CASE(64, 16)
    SOF_CASE(32, 16)
    SOF_CASE(128, 16)
    SOF_CASE(64, 8)
    SOF_CASE(64, 32)
    SOF_CASE(32, 8)
    SOF_CASE(32, 32)
#undef SOF_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_composite_fwd(const CompositeParams &p, int total_tiles, int tile, int chunk, int reorder_k,
                                 cudaStream_t s) {
    return dispatch<false>(p, total_tiles, tile, chunk, reorder_k, s);
}

cudaError_t launch_composite_bwd(const CompositeParams &p, int total_tiles, int tile, int chunk, int reorder_k,
                                 cudaStream_t s) {
    return dispatch<true>(p, total_tiles, tile, chunk, reorder_k, s);
}

}  // namespace sof
