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
// A pixel whose buffer would overflow is abandoned by the main kernel and redone by a second pass
// of it with a 64-entry buffer (only the overflowed pixels of a tile take part); what overflows
// that too is listed (a tile's pixels together) and recomputed exactly by k_composite_fallback (one
// warp per pixel, a sorted buffer of up to kFbCap hits in shared memory), so the result is exact
// for any buffer size.
//
// The backward replays the identical decisions front to back (the same evaluation code runs),
// using the forward's final sums for the contributions of later hits (App. C.1 uses the same
// front-to-back pattern), and accumulates per-record gradients with float4 atomics.
#pragma once

#include <limits.h>
#include <math.h>

#include <algorithm>

#include "record.cuh"
#include "sof_internal.cuh"

namespace sof {
namespace {

constexpr float kInf = 3.402823466e38f;
constexpr int kGradVals = 22;     // gradient values per hit, in the order of the record gradient

// A tile's sorted stream holds one 64-bit word per record: depth key bits << 32 | record index.
__device__ __forceinline__ float pair_key(unsigned long long w) { return __uint_as_float((unsigned)(w >> 32)); }
__device__ __forceinline__ unsigned pair_rec(unsigned long long w) { return (unsigned)w; }

// Pixel of thread tid within its TILE x TILE tile (TILE = 8, 16 or 32): warp w covers the 8x4 block
// at ((w % (TILE / 8)) * 8, (w / (TILE / 8)) * 4), lanes row-major inside it. Compact warp blocks
// let a whole warp skip a record whose pixel bounding box misses its block.
template <int TILE>
__device__ __forceinline__ int tile_px(int tid) { return ((tid >> 5) % (TILE / 8)) * 8 + (tid & 7); }
template <int TILE>
__device__ __forceinline__ int tile_py(int tid) { return ((tid >> 5) / (TILE / 8)) * 4 + ((tid >> 3) & 3); }

// Bits of a thread index within a tile in the overflow lists' (tile << bits | thread) codes.
template <int TILE>
constexpr int tid_bits() { return TILE == 8 ? 6 : (TILE == 16 ? 8 : 10); }

// One of kGradCopies copies of the gradient of record r, chosen by tile (spreads the atomics of
// large Gaussians over several L2-resident addresses); copies are indexed by the record's rank
// among the records with tiles. Null beyond the capacity (counted as dropped by the compaction).
__device__ __forceinline__ float4 *grad_slot(const CompositeParams &p, unsigned r) {
    const int k = p.vis_pos[r];
    return k < p.vis_cap ? p.rgrad + ((size_t)k * kGradCopies + (blockIdx.x & (kGradCopies - 1))) * kGradF4
                         : nullptr;
}

// The replay lists are [tile][k][pixel of the tile]: entry k of a pixel is TILE * TILE words after
// entry k - 1.
template <int TILE>
__device__ __forceinline__ unsigned *list_of(const CompositeParams &p, int gtile, int tid) {
    return p.hit_list ? p.hit_list + (size_t)gtile * p.list_cap * (TILE * TILE) + tid : nullptr;
}

// Backward state of a pixel. With the final sums of the forward, the loss gradient reaching a hit
// from the hits behind it is a scalar: G_final - G_acc, where G = gC.C + gD.D + gN.N.
struct PixelGrad {
    float gC[3], gN[3], gD;
    float gX;       // dL/d(exact depth) + dL/d(median depth): both move with t* of the crossing hit
    float G_final;  // gC.C_final + gD D_final + gN.N_final (background excluded)
    float G_acc;    // the same sum over the hits composited so far, this one included
    float K_bg;     // (dL/dO - gC.bg) T_final: the background term of every hit
};

// NDC planes of the distortion and extent losses (Sec. 3.3): NDC(t) = F (t - N) / ((F - N) t)
constexpr float kNdcN = 0.2f, kNdcF = 100.f;
constexpr float kNdcC = kNdcN * kNdcF / (kNdcF - kNdcN);  // NDC'(t) t^2
// NDC(t) with the fast division (t is a hit's depth, beyond the near plane)
__device__ __forceinline__ float ndc_depth(float t) { return __fdividef(kNdcF * (t - kNdcN), (kNdcF - kNdcN) * t); }

// Extent term e = eps / t*^2 of a hit (App. C.2): eps = |d'| sqrt((E^2 - m) / A'), with the ray's
// Mahalanobis distance m = N / A', E^2 = 2 ln(255 o) kept in the record and t* = t*' |d'|.
__device__ __forceinline__ float extent_term(const RecEval &q, float E2, float tp, float dnorm) {
    const float rA = rec_rcp(q.A);
    const float m = __fmul_rn(q.N, rA);
    const float x = fmaxf(E2 - m, 0.f);
    const float t = __fmul_rn(tp, dnorm);
    return __fdividef(dnorm * sqrtf(x * rA), t * t);
}

// Loss state of a pixel (only in the LOSS instances). Forward: the sums of w d, w d^2 and w e
// over the composited hits (d = NDC(t*), e = eps / t*^2). Backward: the forward's final sums and
// the same sums over the hits replayed so far (with the sum of w in `dist`), with the upstream
// gradients of the two loss channels.
// The pair sum depends only on differences of d, so d is taken relative to the first composited
// hit's (dref): the prefix sums stay small and FP32 keeps their differences.
struct PixelLoss {
    float d1, d2, e, dist, dref;  // sums (d relative to dref); dist: the backward's sum of w
    float fA, fD1, fD2, fE, g_dist, g_ext;  // backward: finals and upstream gradients
};

// Per-pixel compositing state shared by the main kernel and the fallback. NT: pixels per tile (the
// stride of the replay list). LOSS: also the distortion and extent losses (Sec. 3.3, App. C).
template <bool BWD, int NT, bool LOSS = false>
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
    unsigned *lst;  // forward: this pixel's replay list (entry k at lst[k * NT]), or null
    int lcap;
    PixelGrad pg;
    PixelLoss pl;

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
        lst = nullptr;
        lcap = 0;
        if (LOSS) {
            pl.d1 = pl.d2 = pl.e = pl.dist = pl.dref = 0.f;
            if (BWD) {
                const float4 fs = p.loss_sums[pix];
                pl.fA = p.opacity[pix];
                pl.fD1 = fs.x;
                pl.fD2 = fs.y;
                pl.fE = fs.z;
                pl.dref = fs.w;
                pl.g_dist = p.d_distortion ? p.d_distortion[pix] : 0.f;
                pl.g_ext = p.d_extent ? p.d_extent[pix] * kNdcC : 0.f;
            }
        }
        if (BWD) {
            float gfin = 0.f, gbg = 0.f;
            const float Tf = 1.f - p.opacity[pix];
            for (int c = 0; c < 3; ++c) {
                pg.gC[c] = p.d_color ? p.d_color[cbase + (long long)c * HW] : 0.f;
                pg.gN[c] = p.d_normal ? p.d_normal[cbase + (long long)c * HW] : 0.f;
                const float Cf = p.color[cbase + (long long)c * HW] - Tf * p.bg[c];
                gfin = fmaf(pg.gC[c], Cf, fmaf(pg.gN[c], p.normal[cbase + (long long)c * HW], gfin));
                gbg = fmaf(pg.gC[c], p.bg[c], gbg);
            }
            pg.gD = p.d_depth ? p.d_depth[pix] : 0.f;
            pg.gX = (p.d_exact ? p.d_exact[pix] : 0.f) + (p.d_median ? p.d_median[pix] : 0.f);
            pg.G_final = fmaf(pg.gD, p.depth[pix], gfin);
            pg.G_acc = 0.f;
            pg.K_bg = ((p.d_opacity ? p.d_opacity[pix] : 0.f) - gbg) * Tf;
        }
    }

    // Composite the next hit in order (t*' = tp) of record r; returns false if the
    // hit stops the pixel instead. The record's float4 field f is at rec[f * rs] (shared-memory
    // window: rs = window size; global: rs = 1). Backward: the hit's gradients go out as float4
    // atomics to one of the record's gradient copies, from the thread selected by `emit` (the
    // fallback runs a pixel on a whole warp), or, with gout, into gout[0..kGradVals) for the caller
    // to reduce. HAVE_E: the forward's extent term of the hit is given (e_hit), not re-evaluated.
    template <bool HAVE_E = false>
    __device__ __forceinline__ bool composite(const CompositeParams &p, float tp, float a, unsigned r,
                                              const float4 *rec, int rs, bool emit, float *gout = nullptr,
                                              float e_hit = 0.f) {
        const float t = __fmul_rn(tp, dnorm);  // Euclidean t*
        const float Tn = __fmul_rn(T, __fsub_rn(1.f, a));
        if (Tn < p.t_stop) {
            done = true;
            return false;
        }
        const float w = __fmul_rn(a, T);
        const float4 q5 = rec[5 * rs], q6 = rec[6 * rs];
        const float rgb[3] = {q5.y, q5.z, q5.w}, nr[3] = {q6.x, q6.y, q6.z};
        const bool is_cross = !crossed && T > 0.5f && Tn <= 0.5f;
        if (!BWD) {
            for (int c = 0; c < 3; ++c) {
                C[c] = fmaf(w, rgb[c], C[c]);
                Nn[c] = fmaf(w, nr[c], Nn[c]);
            }
            D = fmaf(w, t, D);
            if (LOSS) {
                // distortion: the sums of w d and w d^2 (the pair sum follows from the final sums);
                // extent: sum_i w_i eps_i / t_i^2 (App. C.1, C.2)
                if (cnt == 0) pl.dref = ndc_depth(t);
                const float dn = ndc_depth(t) - pl.dref;
                pl.d1 = fmaf(w, dn, pl.d1);
                pl.d2 = fmaf(w, dn * dn, pl.d2);
                float e = e_hit;
                if (!HAVE_E) {
                    const float4 q0 = rec[0];
                    const RecEval q = rec_eval(q0, rec[rs], rec[2 * rs], rec[3 * rs], rec[4 * rs], q5, fpx - q0.x,
                                               fpy - q0.y);
                    e = extent_term(q, q6.w, tp, dnorm);
                }
                pl.e = fmaf(w, e, pl.e);
            }
            if (lst && emit && cnt < lcap) lst[(size_t)cnt * NT] = r;
            if (is_cross) {
                crossed = true;
                r_cross = r;
                T_cross = T;
                t_cross = t;
            }
        } else {
            if (is_cross) crossed = true;
            const float dLdt = w * pg.gD + (is_cross ? pg.gX : 0.f);
            const float inv = __fdividef(1.f, 1.f - a);  // 1 - a >= 1 - kAlphaMax
            const float front = pg.gC[0] * rgb[0] + pg.gC[1] * rgb[1] + pg.gC[2] * rgb[2] + pg.gD * t +
                                pg.gN[0] * nr[0] + pg.gN[1] * nr[1] + pg.gN[2] * nr[2];
            pg.G_acc = fmaf(w, front, pg.G_acc);
            const float behind = pg.G_final - pg.G_acc;
            // dL/dalpha = T front - (behind - K_bg) / (1 - alpha)
            float dLda = T * front - (behind - pg.K_bg) * inv;
            // re-evaluate the record at this pixel (same arithmetic as the test)
            const float4 q0 = rec[0];
            const RecEval q = rec_eval(q0, rec[rs], rec[2 * rs], rec[3 * rs], rec[4 * rs], q5, fpx - q0.x, fpy - q0.y);
            const float rA = rec_rcp(q.A);
            const float m = __fmul_rn(q.N, rA);
            float dLdt_all = dLdt, dLdm_x = 0.f, dLdA_x = 0.f, dLdo_x = 0.f;
            if (LOSS) {
                // distortion (App. C.1): dL/dw_k = d_k^2 A + D2 - 2 d_k D1 with the final sums; the
                // hits behind k add -(sum_{i>k} w_i dL/dw_i) / (1 - alpha_k), that sum taken from the
                // finals minus the sums so far; dL/dd_k = 2 w_k (d_k A - D1)
                const float dn = ndc_depth(t) - pl.dref;
                const float gk = dn * dn * pl.fA + pl.fD2 - 2.f * dn * pl.fD1;
                pl.d1 = fmaf(w, dn, pl.d1);
                pl.d2 = fmaf(w, dn * dn, pl.d2);
                pl.dist += w;  // the weights so far
                const float S = pl.fA * (pl.fD2 - pl.d2) + pl.fD2 * (pl.fA - pl.dist) - 2.f * pl.fD1 * (pl.fD1 - pl.d1);
                dLda += pl.g_dist * (T * gk - S * inv);
                dLdt_all += pl.g_dist * 2.f * w * (dn * pl.fA - pl.fD1) * __fdividef(kNdcC, t * t);
                // extent (App. C.2): e = eps / t^2, eps = |d'| sqrt((E^2 - m) / A'), E^2 = 2 ln(255 o)
                const float x = q6.w - m;  // E^2 (Eq. 3) kept in the record
                const float e = x > 0.f ? __fdividef(dnorm * sqrtf(x * rA), t * t) : 0.f;
                pl.e = fmaf(w, e, pl.e);
                dLda += pl.g_ext * (T * e - (pl.fE - pl.e) * inv);
                const float ge = pl.g_ext * w;
                dLdt_all += ge * (-2.f * __fdividef(e, t));
                if (x > 0.f) {
                    const float hx = 0.5f * __fdividef(e, x);
                    dLdm_x = -ge * hx;
                    dLdA_x = ge * (-0.5f * e * rA);
                    dLdo_x = ge * hx * __fdividef(2.f, q0.w);  // through E^2
                }
            }
            const float G = __expf(-0.5f * m);
            const bool clamped = !(__fmul_rn(q0.w, G) < kAlphaMax);
            const float dLdm = (clamped ? 0.f : dLda * (-0.5f * a)) + dLdm_x;
            const float dLdo = (clamped ? 0.f : dLda * G) + dLdo_x;
            const float gNq = dLdm * rA;
            const float gA = -(dLdm * m + dLdt_all * t) * rA + dLdA_x;
            const float god = -dLdt_all * dnorm * rA;
            const float gc1 = 2.f * gNq * q.c1, gc2 = 2.f * gNq * q.c2;
            const float dx = q.dx, dy = q.dy;
            if (gout) {
                const float v[kGradVals] = {gc1, gc2, gc1 * dx, gc2 * dx, gc1 * dy, gc2 * dy, gA, gA * dx,
                                            gA * dy, gA * dx * dx, gA * dx * dy, gA * dy * dy, god, god * dx,
                                            god * dy, dLdo, w * pg.gC[0], w * pg.gC[1], w * pg.gC[2],
                                            w * pg.gN[0], w * pg.gN[1], w * pg.gN[2]};
#pragma unroll
                for (int i = 0; i < kGradVals; ++i) gout[i] = v[i];
            } else if (emit) {
                float4 *gp = grad_slot(p, r);
                if (gp) {
                    atomicAdd(gp + 0, make_float4(gc1, gc2, gc1 * dx, gc2 * dx));
                    atomicAdd(gp + 1, make_float4(gc1 * dy, gc2 * dy, gA, gA * dx));
                    atomicAdd(gp + 2, make_float4(gA * dy, gA * dx * dx, gA * dx * dy, gA * dy * dy));
                    atomicAdd(gp + 3, make_float4(god, god * dx, god * dy, dLdo));
                    atomicAdd(gp + 4, make_float4(w * pg.gC[0], w * pg.gC[1], w * pg.gC[2], w * pg.gN[0]));
                    atomicAdd(gp + 5, make_float4(w * pg.gN[1], w * pg.gN[2], 0.f, 0.f));
                }
            }
        }
        T = Tn;
        ++cnt;
        return true;
    }

    __device__ __forceinline__ void write_outputs(const CompositeParams &p) {
        for (int c = 0; c < 3; ++c) {
            p.color[cbase + (long long)c * HW] = C[c] + T * p.bg[c];
            p.normal[cbase + (long long)c * HW] = Nn[c];
        }
        p.depth[pix] = D;
        p.opacity[pix] = 1.f - T;
        p.n_contrib[pix] = cnt;
        if (p.pix_cnt) p.pix_cnt[pix] = cnt;
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
        if (LOSS) {
            // sum_{j<i} w_i w_j (d_i - d_j)^2 is half the sum over all ordered pairs, W D2 - D1^2 with
            // W = sum_i w_i = 1 - T (the pair sum of the expanded squares, in closed form)
            if (p.distortion) p.distortion[pix] = fmaxf(fmaf(1.f - T, pl.d2, -pl.d1 * pl.d1), 0.f);
            if (p.extent) p.extent[pix] = kNdcC * pl.e;
            p.loss_sums[pix] = make_float4(pl.d1, pl.d2, pl.e, pl.dref);
        }
    }
};

__device__ __forceinline__ int view_of_tile(const CamSet *cs, int gtile) {
    int v = 0;
    while (v + 1 < cs->n_views && cs->cam[v + 1].tile_base <= gtile) ++v;
    return v;
}

// Shared-memory layout of the main kernel: the current chunk of the tile's record stream
// (records addressed by stream position, slot = position mod CHUNK) with keys and indices, and the
// per-pixel pending rings.
template <int TILE, int CHUNK, int K, bool BWD, bool LOSS = false>
struct CompositeSmem {
    static constexpr int NT = TILE * TILE;
    // Ring rows: the pixels whose pending buffers the CTA holds at once. The 64-entry instances at
    // 16x16 tiles hold 128 (their shared memory then fits two CTAs per SM, not one) and take the
    // tile's pixels in sweeps of up to 128; the others hold one per thread.
    static constexpr int RS = (K == 64 && TILE == 16) ? 128 : NT;
    static constexpr int kExch = 0;
    // the second pass's instances (K = 64) also hold the compaction of the pixels they redo
    static constexpr size_t compact_bytes =
        K == 64 ? (size_t)(NT / 32) * sizeof(float4) + (size_t)NT * 4 + (size_t)(NT / 32) * 4 + 16 : 0;
    static constexpr size_t base_bytes = (size_t)7 * CHUNK * sizeof(float4) + (size_t)kExch * sizeof(float) +
                                         (size_t)CHUNK * 12 + (size_t)K * RS * 12 + compact_bytes;
    // Forward loss instances with rings of at most 4096 entries keep each pending hit's extent term
    // (computed where the hit is tested) in a fourth ring array, after the rest; the others
    // re-evaluate the record when the hit is composited.
    static constexpr bool ring_e = LOSS && !BWD && K * NT <= 4096;
    static constexpr size_t bytes = base_bytes + (ring_e ? (size_t)K * NT * 4 : 0);
};

// CTAs per SM the register budget is sized for: 64 registers a thread at every tile size, 80 where
// the forward's loss ring leaves shared memory for three CTAs of 16x16 tiles (BIG)
template <int TILE, bool BWD, bool BIG = false>
constexpr int min_ctas() { return TILE == 32 ? 1 : (TILE == 16 ? (BWD || BIG ? 3 : 4) : (BWD ? 12 : 16)); }

template <int TILE, int CHUNK, int K, bool BWD, bool LOSS = false>
__global__ void __launch_bounds__(TILE *TILE, (K == 64 && TILE == 16)
                                                  ? 2  // shared memory holds two CTAs per SM
                                                  : min_ctas<TILE, BWD, CompositeSmem<TILE, CHUNK, K, BWD, LOSS>::ring_e>())
    k_composite(CompositeParams p) {
    using SM = CompositeSmem<TILE, CHUNK, K, BWD, LOSS>;
    constexpr bool kRingE = SM::ring_e;
    constexpr int NT = SM::NT, RS = SM::RS, W = CHUNK;
    extern __shared__ float4 smem[];
    float4 *wrec = smem;                                              // [7][W]
    float *wkey = reinterpret_cast<float *>(wrec + 7 * W);            // [W]
    unsigned *widx = reinterpret_cast<unsigned *>(wkey + W);          // [W] record index
    float *pend_t = reinterpret_cast<float *>(widx + W);              // [K][RS]
    float *pend_a = pend_t + K * RS;                                  // [K][RS]
    unsigned *pend_p = reinterpret_cast<unsigned *>(pend_a + K * RS); // [K][RS] stream position
    unsigned *wmask = pend_p + K * RS;                                // [W] warps the record may hit
    // second-pass instances only (K = 64): the compaction of the redone pixels
    float4 *s_wbox = reinterpret_cast<float4 *>(wmask + W);  // [NT/32] x0, x1, y0, y1 (empty: x0 > x1)
    int *s_slot = reinterpret_cast<int *>(s_wbox + NT / 32);  // [NT] the pixel of each thread
    int *s_wact = s_slot + NT;                                 // [NT/32] active pixels before warp w
    int *s_nact_p = s_wact + NT / 32;                          // [1] active pixels of the tile
    // forward loss instances: the extent term of each pending hit, [K][NT]
    float *pend_e = reinterpret_cast<float *>(reinterpret_cast<char *>(smem) + SM::base_bytes);

    const int tid = threadIdx.x;
    // The second pass's instances (K = 64) run a resident grid over the tiles the first pass left
    // pixels in (or over every tile, where no list is given); the others take one tile per CTA.
    constexpr bool kLoop = K == 64;
    const bool use_list = kLoop && p.redo_tiles != nullptr && p.pass == 1;
    const int n_work = use_list ? *p.redo_count : (kLoop ? p.cams->total_tiles : 1);
    for (int work = kLoop ? (int)blockIdx.x : 0; work < n_work; work += kLoop ? (int)gridDim.x : 1) {
    if (kLoop) __syncthreads();  // the previous tile is done with shared memory
    const int gtile = use_list ? p.redo_tiles[work] : (kLoop ? work : (int)blockIdx.x);
    const DevCam &cam = p.cams->cam[view_of_tile(p.cams, gtile)];
    const int lt = gtile - cam.tile_base;
    const int tx = lt % cam.tiles_x, ty = lt / cam.tiles_x;
    static_assert(TILE == 8 || TILE == 16 || TILE == 32, "tiles of 8, 16 or 32 pixels");
    // with 32-pixel tiles a second pass's larger buffer does not fit in shared memory: the first
    // pass gives its overflowed and open pixels straight to the per-pixel fallback
    constexpr bool kDirectFallback = TILE == 32;
    int slot = tid;  // the tile's pixel this thread takes (its own, unless the pass compacts them)
    int px = tx * TILE + tile_px<TILE>(tid), py = ty * TILE + tile_py<TILE>(tid);
    const int warp = tid >> 5;
    bool inside = px < cam.W && py < cam.H;

    // Pixels this launch handles. The forward's first pass (p.pass == 0) takes every pixel; its
    // overflowed pixels (mask 1) are redone by a second pass with a larger buffer, whose own
    // overflows (mask 2) go to the per-pixel fallback. The backward takes, in each pass, the
    // pixels that pass completed and whose order was not recorded in full (the others replay).
    // A tile with nothing to do returns before loading any pixel state.
    bool skip = !inside;
    if ((BWD || p.pass) && inside) {
        const long long pix = cam.pix_base + (long long)py * cam.W + px;
        const int m = p.ovf_mask[pix];
        skip = BWD ? (m != p.pass || (p.hit_list && p.pix_cnt[pix] <= p.list_cap)) : (m != 1);
    }
    if ((BWD || p.pass) && __syncthreads_and(skip)) continue;
    // The second pass (and the backward's passes) redoes few pixels of a tile, scattered over its
    // warps: they are compacted into the leading threads, so that the warps that walk the list are
    // full and the others skip it. The warps' pixel bounding boxes decide which records they test.
    // The 64-entry instances always compact, and take the compacted pixels in sweeps of RS.
    const bool compact = kLoop;
    int n_act = NT;
    if (compact) {
        const unsigned bm = __ballot_sync(0xffffffffu, !skip);
        if ((tid & 31) == 0) s_wact[warp] = __popc(bm);
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < NT / 32; ++w) {
                const int c = s_wact[w];
                s_wact[w] = tot;
                tot += c;
            }
            *s_nact_p = tot;
        }
        __syncthreads();
        if (!skip) s_slot[s_wact[warp] + __popc(bm & ((1u << (tid & 31)) - 1u))] = tid;
        __syncthreads();
        n_act = *s_nact_p;
    }
    const int n_sweeps = compact ? (n_act + RS - 1) / RS : 1;
    int sweep_f = 0;          // (thread 0) pixels of the tile's earlier sweeps left to the next pass
    bool sweep_open = false;  // (thread 0) whether an earlier sweep asks for the rest of the list
    for (int sw = 0; sw < n_sweeps; ++sw) {
    if (compact) {
        if (sw) __syncthreads();  // the previous sweep is done with the window and the boxes
        const int ci = sw * RS + tid;
        const bool act = tid < RS && ci < n_act;
        slot = act ? s_slot[ci] : tid;
        px = tx * TILE + tile_px<TILE>(slot);
        py = ty * TILE + tile_py<TILE>(slot);
        inside = act;  // the compacted pixels are inside the image
        skip = !act;
        // the bounding box of the warp's pixels
        const int bx0 = __reduce_min_sync(0xffffffffu, act ? px : INT_MAX);
        const int bx1 = __reduce_max_sync(0xffffffffu, act ? px : INT_MIN);
        const int by0 = __reduce_min_sync(0xffffffffu, act ? py : INT_MAX);
        const int by1 = __reduce_max_sync(0xffffffffu, act ? py : INT_MIN);
        if ((tid & 31) == 0) s_wbox[warp] = make_float4((float)bx0, (float)bx1, (float)by0, (float)by1);
        __syncthreads();
    }
    const int2 range = p.ranges[gtile];
    // The first pass reads the sorted front of the tile's list; the key that follows it is a lower
    // bound of every key after the front. The second pass does too, unless a pixel of the tile
    // outlived the front in the first pass (the rest of the list is then sorted).
    const bool front_only = p.prefix_end != nullptr && (p.pass == 0 || !(p.tile_flag[gtile] & kTileOpen));
    const int y_end = front_only ? p.prefix_end[gtile] : range.y;
    // the key after the front, read where it is needed (it is not kept live through the loop)
    auto end_key = [&]() { return front_only ? p.prefix_key[gtile] : kInf; };
    Pixel<BWD, TILE * TILE, LOSS> st;
    st.init(p, cam, inside ? px : 0, inside ? py : 0);
    st.done = skip;
    bool ovf = false;
    if (!BWD) {
        st.lst = list_of<TILE>(p, gtile, slot);
        st.lcap = p.list_cap;
    }

    // pending ring [head, head + pcount) sorted by (t*', record)
    int head = 0, pcount = 0;
    float head_t = kInf, last_t = -kInf;
    bool inexact = false;
    unsigned n_tests = 0, n_hits = 0, n_below = 0;
    int wb = 0;  // first stream position still in the window

    // Pop the smallest pending hit and composite it. Backward: returns whether the lane produced
    // gradients (written to its exchange row) for record *r_out.
    auto pop = [&](unsigned *r_out) -> bool {
        const int sl = head * RS + tid;
        const float t = pend_t[sl], a = pend_a[sl];
        const unsigned pos = pend_p[sl];
        head = (head + 1) & (K - 1);
        --pcount;
        head_t = pcount > 0 ? pend_t[head * RS + tid] : kInf;
        last_t = t;
        const float e = kRingE ? pend_e[sl] : 0.f;
        if ((int)pos >= wb) {
            const int slot = (int)(pos % (unsigned)W);
            *r_out = widx[slot];
            return st.template composite<kRingE>(p, t, a, widx[slot], wrec + slot, W, true, nullptr, e);
        }
        const unsigned r = pair_rec(p.pairs[range.x + pos]);
        *r_out = r;
        return st.template composite<kRingE>(p, t, a, r, p.records + (size_t)r * kRecF4, 1, true, nullptr, e);
    };

    auto insert = [&](float t, float a, unsigned pos, float e) {
        if (t < last_t) inexact = true;  // arrives behind a hit already composited
        if (pcount == K) {
            if (!p.approx) {
                // the buffer is full: leave this pixel to the exact fallback
                ovf = true;
                st.done = true;
                return;
            }
            // opt-in approximate order: the buffer acts as a sort window of K hits; its nearest
            // hit is composited to make room, even if a later record could still hit nearer
            unsigned r;
            pop(&r);
            if (st.done) return;
        }
        int q = pcount;
        while (q > 0) {
            const int sl = ((head + q - 1) & (K - 1)) * RS + tid;
            const float tt = pend_t[sl];
            // ties in t*' go by record index, i.e. by Gaussian index within the view
            if (tt < t || (tt == t && pair_rec(p.pairs[range.x + pend_p[sl]]) < pair_rec(p.pairs[range.x + pos])))
                break;
            const int dl = ((head + q) & (K - 1)) * RS + tid;
            pend_t[dl] = tt;
            pend_a[dl] = pend_a[sl];
            pend_p[dl] = pend_p[sl];
            if (kRingE) pend_e[dl] = pend_e[sl];
            --q;
        }
        const int dl = ((head + q) & (K - 1)) * RS + tid;
        pend_t[dl] = t;
        pend_a[dl] = a;
        pend_p[dl] = pos;
        if (kRingE) pend_e[dl] = e;
        ++pcount;
        if (q == 0) head_t = t;
    };

    // test record j of the chunk staged at slot s
    auto test = [&](int s, int j, int base) {
        const float4 r0 = wrec[s], r1 = wrec[W + s], r2 = wrec[2 * W + s], r3 = wrec[3 * W + s];
        const float4 r4 = wrec[4 * W + s], r5 = wrec[5 * W + s];
        const RecEval q = rec_eval(r0, r1, r2, r3, r4, r5, st.fpx - r0.x, st.fpy - r0.y);
        if (q.N <= __fmul_rn(r0.z, q.A)) {
            float tp, a;
            if (rec_hit(q, r0, r2, st.dnorm, p.near_plane, tp, a)) {
                ++n_hits;
                n_below += (tp < wkey[s]);
                float e = 0.f;
                if (kRingE) e = extent_term(q, wrec[6 * W + s].w, tp, st.dnorm);
                insert(tp, a, (unsigned)(base - range.x + j), e);
            }
        }
    };

    int base = range.x;  // after the loop: the end of the last staged chunk (capped at y_end)
    for (; base < y_end; base += CHUNK) {
        const int n = min(CHUNK, y_end - base);
        __syncthreads();
        for (int i = tid; i < n; i += NT) {
            const unsigned long long pr = p.pairs[base + i];
            widx[i] = pair_rec(pr);
            wkey[i] = pair_key(pr);
        }
        __syncthreads();
        // the records, four pieces a record, each one 256-bit load: fields 0-5 into the window, and
        // field 6 with the pixel bounding box (field 7), which says which warps' pixels the record
        // may hit: the warps' 8x4 blocks, or the boxes of the compacted pixels
        for (int i = tid; i < n * 4; i += NT) {
            const int j = i >> 2, f = 2 * (i & 3);
            float4 a, bb;
            ld_rec_pair(p.records + (size_t)widx[j] * kRecF4 + f, a, bb);
            wrec[f * W + j] = a;
            if (f < 6) {
                wrec[(f + 1) * W + j] = bb;
                continue;
            }
            unsigned mk = 0u;
            if (compact) {
#pragma unroll
                for (int w = 0; w < NT / 32; ++w) {
                    const float4 wb4 = s_wbox[w];
                    mk |= (unsigned)!(bb.y < wb4.x || bb.x > wb4.y || bb.w < wb4.z || bb.z > wb4.w) << w;
                }
            } else {
#pragma unroll
                for (int w = 0; w < NT / 32; ++w) {
                    const float x0 = (float)(tx * TILE + (w % (TILE / 8)) * 8);
                    const float y0 = (float)(ty * TILE + (w / (TILE / 8)) * 4);
                    mk |= (unsigned)!(bb.y < x0 || bb.x > x0 + 7.f || bb.w < y0 || bb.z > y0 + 3.f) << w;
                }
            }
            wmask[j] = mk;
        }
        const float tlo_after = (base + n < y_end) ? pair_key(p.pairs[base + n]) : end_key();
        if (!BWD && tid < 32) {
            // the merge needs non-decreasing keys within the tile's stream (checked by warp 0)
            bool bad = tid == 0 && tlo_after < wkey[n - 1];
            for (int i = 1 + tid; i < n; i += 32) bad |= wkey[i] < wkey[i - 1];
            if (__any_sync(0xffffffffu, bad) && tid == 0) atomicAdd(&p.status->n_unsorted, 1ull);
        }
        wb = base - range.x;
        __syncthreads();
        if (!st.done) {
            int j = 0;
            for (; j < n; ++j) {
                // the whole warp skips a record whose bounding box misses its block: no test, and
                // no drain needed (pending hits simply wait for the next drain)
                if (!((wmask[j] >> warp) & 1u)) continue;
                test(j, j, base);
                if (st.done) break;
                const float tn = (j + 1 < n) ? wkey[j + 1] : tlo_after;
                unsigned r;
                while (pcount > 0 && head_t < tn) {
                    pop(&r);
                    if (st.done) break;
                }
                if (st.done) break;
            }
            n_tests += (unsigned)min(j + 1, n);
        }
        if (__syncthreads_and(st.done)) {
            base += CHUNK;
            break;
        }
    }
    const int read_end = min(base, y_end);
    const float ek = end_key();
    {
        unsigned r;
        if (ek == kInf) {
            while (!st.done && pcount > 0) pop(&r);
        } else {
            // only the hits below every key after the front are final
            while (!st.done && pcount > 0 && head_t < ek) pop(&r);
        }
    }
    // still open where the front ends: redone by the next pass over the whole list
    const bool open = !BWD && !st.done && ek < kInf;

    if (!BWD) {
        // the tile's overflowed pixels take consecutive entries of the list, so that the fallback
        // works on one tile's records with neighbouring warps
        __shared__ int s_wcnt[NT / 32], s_base;
        const bool active = !skip;
        const bool f = active && (ovf || open);
        const bool any_open = __syncthreads_or(open);
        const unsigned fb = __ballot_sync(0xffffffffu, f);
        if ((tid & 31) == 0) s_wcnt[tid >> 5] = __popc(fb);
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < NT / 32; ++w) {
                const int c = s_wcnt[w];
                s_wcnt[w] = tot;
                tot += c;
            }
            s_base = tot ? atomicAdd((p.pass || kDirectFallback) ? p.ovf_count2 : p.ovf_count, tot) : 0;
            // tiles whose rest of the list the next pass needs sorted: the first pass's open tiles;
            // in the second pass, every tile of a fallback pixel that still reads the front only
            sweep_f += tot;
            sweep_open = sweep_open || (p.pass ? (tot && front_only) : any_open);
            if (sw == n_sweeps - 1) {  // each tile is listed once, after its last sweep
                if (!p.pass && sweep_f && p.redo_tiles) p.redo_tiles[atomicAdd(p.redo_count, 1)] = gtile;
                if (p.open_tiles[0] && sweep_open) {
                    if (!p.pass) p.tile_flag[gtile] = kTileOpen;
                    p.open_tiles[p.pass][atomicAdd(p.open_count[p.pass], 1)] = gtile;
                }
            }
            if (!p.pass) add_count(p.status, kCntRead, (unsigned long long)(read_end - range.x));
        }
        __syncthreads();
        if (f) {
            const int e = s_base + s_wcnt[tid >> 5] + __popc(fb & ((1u << (tid & 31)) - 1u));
            ((p.pass || kDirectFallback) ? p.ovf_list2 : p.ovf_list)[e] =
                ((unsigned)gtile << tid_bits<TILE>()) | (unsigned)slot;
        }
        if (active) {
            p.ovf_mask[st.pix] = (unsigned char)(p.pass + (f ? (kDirectFallback ? 2 : 1) : 0));
            if (!f) st.write_outputs(p);
        }
    }
    if (inexact) atomicAdd(&p.status->inexact_pixels, 1ull);
    if (!BWD) {
        // work counters (one atomic per warp)
        const bool redo = !skip && (ovf || open);
        unsigned long long a = n_tests, b = n_hits, cc = redo ? 0u : (unsigned)st.cnt, e = n_below;
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
            cc += __shfl_xor_sync(0xffffffffu, cc, o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
        }
        const unsigned n_ovf = __popc(__ballot_sync(0xffffffffu, !skip && ovf));
        const unsigned n_open = __popc(__ballot_sync(0xffffffffu, !skip && !ovf && open));
        if ((tid & 31) == 0) {
            add_count(p.status, kCntTests, a);
            add_count(p.status, kCntHits, b);
            add_count(p.status, kCntComposited, cc);
            if (e) atomicAdd(&p.status->n_below_key, e);
            if (!p.pass && n_ovf) atomicAdd(&p.status->n_forced, (unsigned long long)n_ovf);
            if (n_open) atomicAdd(&p.status->n_open, (unsigned long long)n_open);
        }
    }
    }  // sweeps
    }  // tiles
}

// Exact fallback for pixels whose pending buffer overflowed: one warp per pixel runs the same
// streaming merge with a large buffer in shared memory. It tests the tile's records 32 at a time
// (keys ascending), collects the hits as (t*' bits << 32 | record), sorts the buffer (bitonic), and
// composites the entries below the key of the first record not yet tested -- no later record can
// produce an earlier hit -- keeping the rest for the next round. If a full buffer could make no
// progress, the pixel finishes by plain selection of the next hit in order.
constexpr int kFbWarps = 8;   // neighbouring list entries (one tile's pixels) share a CTA and its L1
constexpr int kFbCap = 1024;

__device__ __forceinline__ bool fb_test(const CompositeParams &p, const float4 *rp, float fpx, float fpy,
                                        float dnorm, float &tp, float &a) {
    const float4 bb = rp[7];  // pixel bounding box: outside it the pre-test cannot pass
    if (fpx < bb.x || fpx > bb.y || fpy < bb.z || fpy > bb.w) return false;
    float4 r0, r1, r2, r3, r4, r5;  // three 256-bit loads
    ld_rec_pair(rp, r0, r1);
    ld_rec_pair(rp + 2, r2, r3);
    ld_rec_pair(rp + 4, r4, r5);
    const RecEval q = rec_eval(r0, r1, r2, r3, r4, r5, fpx - r0.x, fpy - r0.y);
    return q.N <= __fmul_rn(r0.z, q.A) && rec_hit(q, r0, r2, dnorm, p.near_plane, tp, a);
}

template <int TILE, bool BWD, bool LOSS = false>
__global__ void __launch_bounds__(kFbWarps * 32) k_composite_fallback(CompositeParams p) {
    extern __shared__ unsigned long long fbuf[];
    const int lane = threadIdx.x & 31;
    unsigned long long *buf = fbuf + (threadIdx.x >> 5) * kFbCap;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int count = *p.ovf_count2;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int e = warp; e < count; e += n_warps) {
        const unsigned code = p.ovf_list2[e];
        const int gtile = (int)(code >> tid_bits<TILE>()), tid = (int)(code & ((1u << tid_bits<TILE>()) - 1u));
        const DevCam &cam = p.cams->cam[view_of_tile(p.cams, gtile)];
        const int lt = gtile - cam.tile_base;
        const int px = (lt % cam.tiles_x) * TILE + tile_px<TILE>(tid);
        const int py = (lt / cam.tiles_x) * TILE + tile_py<TILE>(tid);
        const int2 range = p.ranges[gtile];
        Pixel<BWD, TILE * TILE, LOSS> st;
        st.init(p, cam, px, py);
        if (BWD && p.hit_list && p.pix_cnt[st.pix] <= p.list_cap) continue;  // replayed instead
        if (!BWD) {
            st.lst = list_of<TILE>(p, gtile, tid);
            st.lcap = p.list_cap;
        }
        unsigned long long last = 0ull;  // (t*' bits << 32 | record) of the last composited hit
        int cnt = 0, cursor = range.x;
        bool stalled = false;
        auto composite_entry = [&](unsigned long long pk) {
            const unsigned ev = (unsigned)(pk & 0xFFFFFFFFull);
            const unsigned r = ev;
            const float4 *rp = p.records + (size_t)r * kRecF4;
            float tp, a;
            fb_test(p, rp, st.fpx, st.fpy, st.dnorm, tp, a);
            st.composite(p, tp, a, r, rp, 1, lane == 0);
            last = pk;
        };
        while (!st.done) {
            // fill: test records 32 at a time until the buffer could overflow
            while (cursor < range.y && cnt <= kFbCap - 32) {
                const int j = cursor + lane;
                unsigned long long pk = 0ull;
                bool hit = false;
                if (j < range.y) {
                    const unsigned ev = pair_rec(p.pairs[j]);
                    float tp, a;
                    hit = fb_test(p, p.records + (size_t)ev * kRecF4, st.fpx, st.fpy, st.dnorm, tp, a);
                    pk = ((unsigned long long)__float_as_uint(tp) << 32) | ev;
                }
                const unsigned m = __ballot_sync(0xffffffffu, hit);
                if (hit) buf[cnt + __popc(m & lt_mask)] = pk;
                cnt += __popc(m);
                cursor += 32;
            }
            if (cursor > range.y) cursor = range.y;
            const float limit = cursor < range.y ? pair_key(p.pairs[cursor]) : kInf;
            if (cnt == 0) {
                if (cursor >= range.y) break;
                continue;
            }
            // bitonic sort of buf[0, P), padded with the largest key
            int P = 32;
            while (P < cnt) P <<= 1;
            for (int i = cnt + lane; i < P; i += 32) buf[i] = ~0ull;
            __syncwarp();
            for (int k = 2; k <= P; k <<= 1)
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    for (int i = lane; i < P; i += 32) {
                        const int ix = i ^ jj;
                        if (ix > i) {
                            const unsigned long long x = buf[i], y = buf[ix];
                            const bool up = (i & k) == 0;
                            if ((x > y) == up) {
                                buf[i] = y;
                                buf[ix] = x;
                            }
                        }
                    }
                    __syncwarp();
                }
            // composite everything below the next untested key
            int i = 0;
            while (i < cnt && !st.done && __uint_as_float((unsigned)(buf[i] >> 32)) < limit) {
                composite_entry(buf[i]);
                ++i;
            }
            if (st.done) break;
            if (i == 0 && cnt > kFbCap - 32) {
                stalled = true;
                break;
            }
            // keep the rest at the front
            const int rest = cnt - i;
            for (int b = 0; b < rest; b += 32) {
                const unsigned long long v = (b + lane < rest) ? buf[i + b + lane] : 0ull;
                __syncwarp();
                if (b + lane < rest) buf[b + lane] = v;
                __syncwarp();
            }
            cnt = rest;
            if (cursor >= range.y && cnt == 0) break;
        }
        // last resort: select the next hit in (t*', record) order until done
        while (stalled && !st.done) {
            unsigned long long best = ~0ull;
            for (int base = range.x; base < range.y; base += 32) {
                const float kb = pair_key(p.pairs[base]);
                if (best != ~0ull && kb > __uint_as_float((unsigned)(best >> 32))) break;
                const int j = base + lane;
                unsigned long long cand = ~0ull;
                if (j < range.y) {
                    const unsigned ev = pair_rec(p.pairs[j]);
                    float tp, a;
                    if (fb_test(p, p.records + (size_t)ev * kRecF4, st.fpx, st.fpy, st.dnorm, tp, a)) {
                        const unsigned long long pk = ((unsigned long long)__float_as_uint(tp) << 32) | ev;
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
            composite_entry(best);
        }
        if (!BWD && lane == 0) {
            st.write_outputs(p);
            add_count(p.status, kCntComposited, (unsigned long long)st.cnt);
        }
        __syncwarp();
    }
}

// Backward of every pixel whose composite order the forward recorded in full: the pixel walks its
// list front to back, re-evaluates each hit with the forward's arithmetic (so T, w and the 0.5
// crossing are bit-identical) and computes the hit's gradients. No tests, no merge.
//
// Warp-reduced atomics: at each step the warp's lanes (an 8x4 pixel block) hold hits of only a
// few distinct records. Lanes are grouped by record (match_any), each group is given a contiguous
// range of positions, the values are written to shared memory in that order, 22 lanes sum one
// value each along the segments, and one lane per group sends the sums with six float4 atomics.
// Row of the per-warp reduction scratch: 32 positions plus 4 of padding, so that a row is read as
// float4s and lane c's scalar accesses at column q fall on bank (4c + q) mod 32.
constexpr int kRedStride = 36;
// Row of the per-warp segment sums, [segment][value]: a multiple of 4 floats, 4 modulo 32, so that
// the groups' last lanes read their sums as float4s from distinct banks (up to 8 segments per
// quarter warp) and the walking lanes write one segment's values to consecutive banks.
constexpr int kSegStride = 36;
// Shared memory of the replay: per warp the reduction rows and the segment sums (dynamic: above
// the 48 KB of static shared memory).
constexpr size_t kReplaySmem = (size_t)8 * (kGradVals * kRedStride + 32 * kSegStride) * sizeof(float);

// CTAs of 256 threads cover consecutive (tile, pixel) slots, so a warp is one 8x4 block of a tile
// at every tile size.
template <int TILE, bool LOSS>
__device__ __forceinline__ void replay_walk(const CompositeParams &p) {
    constexpr int NT = TILE * TILE;
    extern __shared__ __align__(16) float replay_smem[];  // [8][kGradVals][kRedStride], [8][32][kSegStride]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long slot = (long long)blockIdx.x * 256 + threadIdx.x;
    const int gtile = (int)(slot / NT), tid = (int)(slot % NT);
    if (gtile >= p.cams->total_tiles) return;  // whole warps: NT is a multiple of 32
    const DevCam &cam = p.cams->cam[view_of_tile(p.cams, gtile)];
    const int lt = gtile - cam.tile_base;
    const int px = (lt % cam.tiles_x) * TILE + tile_px<TILE>(tid), py = (lt / cam.tiles_x) * TILE + tile_py<TILE>(tid);
    const bool inside = px < cam.W && py < cam.H;
    Pixel<true, NT, LOSS> st;
    st.init(p, cam, inside ? px : 0, inside ? py : 0);
    int n = inside ? p.pix_cnt[st.pix] : 0;
    if (n > p.list_cap) n = 0;  // re-merged by k_composite
    const unsigned *lst = list_of<TILE>(p, gtile, tid);
    float *wr = replay_smem + warp * (kGradVals * kRedStride);
    float *ws = replay_smem + 8 * (kGradVals * kRedStride) + warp * (32 * kSegStride);
    const unsigned lt_mask = (1u << lane) - 1u;
    const int n_max = __reduce_max_sync(0xffffffffu, (unsigned)n);
    // software pipeline: the list entries three hits ahead are in registers, so a hit's record
    // loads do not wait for its list load
    unsigned r_next = n > 0 ? lst[0] : 0u, r_next2 = n > 1 ? lst[NT] : 0u;
    unsigned r_next3 = n > 2 ? lst[2 * NT] : 0u;
    for (int k = 0; k < n_max; ++k) {
        const bool act = k < n;
        float v[kGradVals];
        unsigned r = 0xFFFFFFFFu;
        if (act) {
            r = r_next;
            r_next = r_next2;
            r_next2 = r_next3;
            if (k + 3 < n) r_next3 = lst[(size_t)(k + 3) * NT];
            // the record's first seven float4 in three 256-bit loads and one 128-bit load: each
            // load instruction costs one L1 wavefront per distinct record in the warp
            const float4 *rp = p.records + (size_t)r * kRecF4;
            float4 lr[7];
            ld_rec_pair(rp, lr[0], lr[1]);
            ld_rec_pair(rp + 2, lr[2], lr[3]);
            ld_rec_pair(rp + 4, lr[4], lr[5]);
            lr[6] = __ldg(rp + 6);
            const RecEval q = rec_eval(lr[0], lr[1], lr[2], lr[3], lr[4], lr[5], st.fpx - lr[0].x, st.fpy - lr[0].y);
            float tp, a;
            rec_hit(q, lr[0], lr[2], st.dnorm, p.near_plane, tp, a);  // a recorded hit: the test passed
            st.composite(p, tp, a, r, lr, 1, true, v);
        }
        // group the active lanes by record; inactive lanes form no group
        const unsigned amask = __ballot_sync(0xffffffffu, act);
        const unsigned grp = __match_any_sync(0xffffffffu, r) & amask;
        const int n_act = __popc(amask);
        const bool leader = act && (__ffs(grp) - 1) == lane;
        const unsigned lmask = __ballot_sync(0xffffffffu, leader);
        if (__popc(lmask) == n_act) {
            // all records distinct: nothing to combine
            float4 *gp = act ? grad_slot(p, r) : nullptr;
            if (gp) {
                atomicAdd(gp + 0, make_float4(v[0], v[1], v[2], v[3]));
                atomicAdd(gp + 1, make_float4(v[4], v[5], v[6], v[7]));
                atomicAdd(gp + 2, make_float4(v[8], v[9], v[10], v[11]));
                atomicAdd(gp + 3, make_float4(v[12], v[13], v[14], v[15]));
                atomicAdd(gp + 4, make_float4(v[16], v[17], v[18], v[19]));
                atomicAdd(gp + 5, make_float4(v[20], v[21], 0.f, 0.f));
            }
            continue;
        }
        // segment of each group: groups ordered by leader lane, members by lane
        unsigned sz = leader ? (unsigned)__popc(grp) : 0u, incl = sz;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const unsigned start = __shfl_sync(0xffffffffu, incl - sz, act ? __ffs(grp) - 1 : lane);
        const int pos = (int)start + __popc(grp & lt_mask);
        const bool seg_end = act && (grp >> lane) == 1u;  // last member of its group
        const unsigned ends = __reduce_or_sync(0xffffffffu, seg_end ? (1u << pos) : 0u);
        if (act) {
#pragma unroll
            for (int c = 0; c < kGradVals; ++c) wr[c * kRedStride + pos] = v[c];
        }
        __syncwarp();
        if (lane < kGradVals) {
            // the segment sums along the row, four positions per shared-memory load (the last
            // position is a segment's end, so what follows it in the last float4 is never kept)
            float acc = 0.f;
            const float *row = wr + lane * kRedStride;
            float *out = ws + lane;  // value `lane` of segment sg at out[sg * kSegStride]
            int sg = 0;
            for (int q = 0; q < n_act; q += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(row + q);
                const unsigned e = ends >> q;
                acc += v.x;
                if (e & 1u) {
                    out[kSegStride * sg++] = acc;
                    acc = 0.f;
                }
                acc += v.y;
                if (e & 2u) {
                    out[kSegStride * sg++] = acc;
                    acc = 0.f;
                }
                acc += v.z;
                if (e & 4u) {
                    out[kSegStride * sg++] = acc;
                    acc = 0.f;
                }
                acc += v.w;
                if (e & 8u) {
                    out[kSegStride * sg++] = acc;
                    acc = 0.f;
                }
            }
        }
        __syncwarp();
        if (seg_end) {
            const int sg = __popc(ends & ((1u << pos) - 1u));  // the segments before this one
            const float4 *sr = reinterpret_cast<const float4 *>(ws + sg * kSegStride);
            float s_[24];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const float4 x = sr[c];
                s_[4 * c] = x.x;
                s_[4 * c + 1] = x.y;
                s_[4 * c + 2] = x.z;
                s_[4 * c + 3] = x.w;
            }
            float4 *gp = grad_slot(p, r);
            if (gp) {
                atomicAdd(gp + 0, make_float4(s_[0], s_[1], s_[2], s_[3]));
                atomicAdd(gp + 1, make_float4(s_[4], s_[5], s_[6], s_[7]));
                atomicAdd(gp + 2, make_float4(s_[8], s_[9], s_[10], s_[11]));
                atomicAdd(gp + 3, make_float4(s_[12], s_[13], s_[14], s_[15]));
                atomicAdd(gp + 4, make_float4(s_[16], s_[17], s_[18], s_[19]));
                atomicAdd(gp + 5, make_float4(s_[20], s_[21], 0.f, 0.f));
            }
        }
        __syncwarp();
    }
    unsigned long long tot = (unsigned)n;
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0 && tot) add_count(p.status, kCntReplayed, tot);
}

// The replay kernels. Three CTAs per SM: the plain instance fits them by itself (79 registers); the
// loss-channel instance is bounded to them (80 registers instead of 90, which fit two).
template <int TILE>
__global__ void __launch_bounds__(256) k_composite_replay(CompositeParams p) { replay_walk<TILE, false>(p); }
template <int TILE>
__global__ void __launch_bounds__(256, 3) k_composite_replay_loss(CompositeParams p) { replay_walk<TILE, true>(p); }

// Launches the replay with its dynamic shared memory (the attribute is set on first use).
template <int TILE, bool LOSS>
cudaError_t launch_replay_instance(const CompositeParams &p, unsigned grid, cudaStream_t s) {
    auto kern = LOSS ? k_composite_replay_loss<TILE> : k_composite_replay<TILE>;
    static bool configured = false;
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute((const void *)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kReplaySmem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    kern<<<grid, 256, kReplaySmem, s>>>(p);
    return cudaGetLastError();
}

// Opacity field at the exact depth on each pixel's ray (Sec. 3.3 "Direct Opacity Field
// Supervision": L_opa = (O_N(c + t d) - 0.5)^2 with t the exact depth), over the hits the pixel
// composited, from the forward's recorded order: O = 1 - prod (1 - alpha_i(t_eval)),
// t_eval = min(t*_i, t), a hit counting where alpha_i(t_eval) >= 1/255 (Eqs. 11-12). Hits behind
// the point are evaluated off their peak: the ray's Mahalanobis distance there is
// m + A' (t' - t*')^2 (t' = t / |d'|, the record's pixel-plane units). The exact depth is taken
// as given (not differentiated). Pixels without a 0.5 crossing, or with more hits than the
// recorded lists hold, get -1 and no gradient.
// BWD: dL/dalpha_i = g (1 - O) / (1 - alpha_i), g the upstream gradient, chained through m, A',
// t*' and o into the record gradient (direct float4 atomics: an opt-in channel).
template <int TILE, bool BWD>
__global__ void __launch_bounds__(256) k_opacity_at_depth(CompositeParams p) {
    constexpr int NT = TILE * TILE;
    const long long slot = (long long)blockIdx.x * 256 + threadIdx.x;
    const int gtile = (int)(slot / NT), tid = (int)(slot % NT);
    if (gtile >= p.cams->total_tiles) return;
    const DevCam &cam = p.cams->cam[view_of_tile(p.cams, gtile)];
    const int lt = gtile - cam.tile_base;
    const int px = (lt % cam.tiles_x) * TILE + tile_px<TILE>(tid), py = (lt / cam.tiles_x) * TILE + tile_py<TILE>(tid);
    if (px >= cam.W || py >= cam.H) return;
    const long long pix = cam.pix_base + (long long)py * cam.W + px;
    const int n = p.pix_cnt[pix];
    const float tx = p.exact_depth[pix];
    if (n > p.list_cap || !(tx > 0.f)) {
        if (!BWD) p.opa[pix] = -1.f;
        return;
    }
    const float g = BWD ? p.d_opa[pix] : 0.f;
    if (BWD && (g == 0.f || !(p.opa[pix] >= 0.f))) return;
    const float uu = ((float)px + 0.5f - cam.cx) / cam.fx, vv = ((float)py + 0.5f - cam.cy) / cam.fy;
    const float dnorm = sqrtf(1.f + uu * uu + vv * vv);
    const float txp = tx / dnorm;  // the point's t' along d' = (u, v, 1)
    const float gP = BWD ? g * (1.f - p.opa[pix]) : 0.f;  // g * prod_all (1 - alpha)
    const unsigned *lst = list_of<TILE>(p, gtile, tid);
    float P = 1.f;
    for (int k = 0; k < n; ++k) {
        const unsigned r = lst[(size_t)k * NT];
        const float4 *rp = p.records + (size_t)r * kRecF4;
        float4 r0, r1, r2, r3, r4, r5;  // three 256-bit loads
        ld_rec_pair(rp, r0, r1);
        ld_rec_pair(rp + 2, r2, r3);
        ld_rec_pair(rp + 4, r4, r5);
        const RecEval q = rec_eval(r0, r1, r2, r3, r4, r5, (float)px - r0.x, (float)py - r0.y);
        const float rA = rec_rcp(q.A);
        const float m = __fmul_rn(q.N, rA);
        const float tp = __fmul_rn(-rec_od(r2, q.dx, q.dy), rA);
        const float dl = tp > txp ? txp - tp : 0.f;  // t_eval' - t*'
        const float qq = fmaf(q.A * dl, dl, m);
        const float G = __expf(-0.5f * qq);
        const float a = fminf(kAlphaMax, r0.w * G);
        if (!(a >= kAlphaMin)) continue;
        if (!BWD) {
            P *= 1.f - a;
            continue;
        }
        if (!(r0.w * G < kAlphaMax)) continue;  // clamped: no gradient through the parameters
        const float dLda = __fdividef(gP, 1.f - a);
        const float dLdq = dLda * (-0.5f * a);
        const float dLdo = dLda * G;
        // qq = m + A' dl^2, dl = t' - t*': through m (N, A'), A' directly, and t*' = -od / A'
        const float dLdm = dLdq;
        const float dLdA_x = dLdq * dl * dl;
        const float dLdtp = dLdq * (-2.f * q.A * dl);  // d qq / d t*'
        const float dLdt = dLdtp / dnorm;               // per Euclidean t*, as the assembly takes it
        const float t = tp * dnorm;
        const float gNq = dLdm * rA;
        const float gA = -(dLdm * m + dLdt * t) * rA + dLdA_x;
        const float god = -dLdt * dnorm * rA;
        const float gc1 = 2.f * gNq * q.c1, gc2 = 2.f * gNq * q.c2;
        const float dx = q.dx, dy = q.dy;
        float4 *gp = grad_slot(p, r);
        if (gp) {
            atomicAdd(gp + 0, make_float4(gc1, gc2, gc1 * dx, gc2 * dx));
            atomicAdd(gp + 1, make_float4(gc1 * dy, gc2 * dy, gA, gA * dx));
            atomicAdd(gp + 2, make_float4(gA * dy, gA * dx * dx, gA * dx * dy, gA * dy * dy));
            atomicAdd(gp + 3, make_float4(god, god * dx, god * dy, dLdo));
        }
    }
    if (!BWD) p.opa[pix] = 1.f - P;
}

template <int TILE, int CHUNK, int K, bool BWD, bool LOSS = false>
cudaError_t launch_t(const CompositeParams &p, int total_tiles, cudaStream_t s) {
    const size_t sm = CompositeSmem<TILE, CHUNK, K, BWD, LOSS>::bytes;
    static bool configured = false;
    static int resident = 0;  // CTAs the whole GPU holds at once
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_composite<TILE, CHUNK, K, BWD, LOSS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        int dev = 0, n_sm = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_composite<TILE, CHUNK, K, BWD, LOSS>,
                                                                 TILE * TILE, sm)) != cudaSuccess)
            return e;
        resident = std::max(1, n_sm * per_sm);
        configured = true;
    }
    note_launches(1);
    // the second pass's instances loop over their tiles: one resident wave
    const int grid = K == 64 ? std::min(total_tiles, resident) : total_tiles;
    k_composite<TILE, CHUNK, K, BWD, LOSS><<<grid, TILE * TILE, sm, s>>>(p);
    return cudaGetLastError();
}

// The fallback reads the overflow count on the device: a fixed grid of 3 CTAs per SM.
template <int TILE, bool BWD, bool LOSS = false>
cudaError_t launch_fb(const CompositeParams &p, cudaStream_t s) {
    constexpr size_t fsm = (size_t)kFbWarps * kFbCap * sizeof(unsigned long long);
    static bool fconfigured = false;
    if (!fconfigured) {
        cudaError_t e = cudaFuncSetAttribute(k_composite_fallback<TILE, BWD, LOSS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
        if (e != cudaSuccess) return e;
        fconfigured = true;
    }
    note_launches(1);
    k_composite_fallback<TILE, BWD, LOSS><<<device_sm_count() * 3, kFbWarps * 32, fsm, s>>>(p);
    return cudaGetLastError();
}

// Instantiated (tile, chunk, buffer) triples; K = 64 serves the second pass at tiles 8 and 16. LOSS:
// the instances with the distortion and extent channels (compiled in their own unit).
template <bool BWD, bool LOSS>
cudaError_t dispatch(const CompositeParams &p, int total_tiles, int tile, int chunk, int k, cudaStream_t s) {
    if (total_tiles <= 0) return cudaSuccess;
#define SOF_CASE(TT, CH, KK) \
    if (tile == TT && chunk == CH && k == KK) return launch_t<TT, CH, KK, BWD, LOSS>(p, total_tiles, s);
    SOF_CASE(16, 64, 16)
    SOF_CASE(16, 32, 16)
    SOF_CASE(16, 128, 16)
    SOF_CASE(16, 64, 8)
    SOF_CASE(16, 64, 32)
    SOF_CASE(16, 32, 8)
    SOF_CASE(16, 32, 32)
    SOF_CASE(16, 32, 64)
    SOF_CASE(16, 64, 64)
    SOF_CASE(16, 128, 64)
    SOF_CASE(8, 64, 16)
    SOF_CASE(8, 64, 32)
    SOF_CASE(8, 64, 64)
    SOF_CASE(32, 64, 8)
    SOF_CASE(32, 64, 16)
#undef SOF_CASE
    return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace sof
