// Layout of the per-(Gaussian, view) record and its per-pixel evaluation, shared by the binning,
// compositing and query kernels so that every path takes bit-identical decisions.
//
// Pixel (px, py) has integer offset (dx, dy) = (px - ia, py - ja) from the anchor pixel
// (ia, ja) (the pixel containing the projected mean; the image centre when the mean does not
// project). With o_g = S^-1 R^T (c - mu) and d_g(d) = S^-1 R^T R_c^T ((px+0.5-cx)/fx,
// (py+0.5-cy)/fy, 1) (Sec. 3.1 "Gaussian Opacity Fields", Eqs. 4-5, R^T since R maps local to world):
//   cross(d) = (c1 + p1 dx + q1 dy, c2 + q2 dy)  = o_g x d_g(d) in an orthonormal basis of the
//                                                  plane normal to o_g
//   d_g(d)   = dga + dx a + dy b                 (evaluated as a 3-vector: conditioning linear,
//                                                  not quadratic, in the anisotropy)
//   A(d)     = |d_g(d)|^2,   od(d) = od0 + odx dx + ody dy = o_g . d_g(d)
// m = |cross|^2 / A = C - B^2/4A (Eq. 10 through Lagrange's identity), and the peak of the ray
// (Eq. 9) lies at t*' = -od/A in camera-z units of d' = (u, v, 1), i.e. t* = t*' |d'|.
//   f4[0] = (ia, ja, e2t, o)        e2t = E^2 (1 + 1e-4): conservative pre-test threshold
//   f4[1] = (c1, c2, p1, q1)
//   f4[2] = (q2, od0, odx, ody)
//   f4[3] = (dga.x, dga.y, dga.z, a.x)
//   f4[4] = (a.y, a.z, b.x, b.y)
//   f4[5] = (b.z, red, green, blue)
//   f4[6] = render: (nx, ny, nz, E^2)    query: (delta_x, delta_y, z_mu hi, z_mu lo)
//   f4[7] = render: (x0, x1, y0, y1) inclusive pixel-index bounding box of the silhouette
//           query: (z_min, proj_ok, 0, 0)
// delta = anchor centre - projected mean (pixels); for the query the peak relative to the mean is
// z_mu - t*' = z_mu d_g(d) . ((dx + delta_x) a + (dy + delta_y) b) / A, which vanishes at the
// mean's projection, so the depth of a point relative to a Gaussian's peak is cancellation-free.
#pragma once

#include "sof_internal.cuh"

namespace sof {

constexpr int kRecStage = 6;  // float4 of a record that the test needs (f4[0..5])

struct RecEval {
    float dx, dy;      // offset from the anchor pixel
    float c1, c2;      // o_g x d_g in the plane basis
    float N, A;        // |cross|^2, |d_g|^2
    float gx, gy, gz;  // d_g
};

// Two consecutive float4 of a record with one 256-bit load through the read-only path. The pair
// must start at an even float4 of a record (records are 128-byte aligned, so it is 32-byte aligned),
// and the records must not change during the kernel.
__device__ __forceinline__ void ld_rec_pair(const float4 *p, float4 &a, float4 &b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Closed-form geometry of one record at offset (dx, dy).
__device__ __forceinline__ RecEval rec_eval(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r3,
                                            const float4 &r4, const float4 &r5, float dx, float dy) {
    RecEval e;
    e.dx = dx;
    e.dy = dy;
    e.c1 = fmaf(r1.z, dx, fmaf(r1.w, dy, r1.x));
    e.c2 = fmaf(r2.x, dy, r1.y);
    e.N = fmaf(e.c1, e.c1, __fmul_rn(e.c2, e.c2));
    e.gx = fmaf(dy, r4.z, fmaf(dx, r3.w, r3.x));
    e.gy = fmaf(dy, r4.w, fmaf(dx, r4.x, r3.y));
    e.gz = fmaf(dy, r5.x, fmaf(dx, r4.y, r3.z));
    e.A = fmaf(e.gx, e.gx, fmaf(e.gy, e.gy, __fmul_rn(e.gz, e.gz)));
    return e;
}

__device__ __forceinline__ float rec_od(const float4 &r2, float dx, float dy) {
    return fmaf(r2.z, dx, fmaf(r2.w, dy, r2.y));
}

// 1 / A' for the Mahalanobis distance m = N / A' and the peak t*' = -od / A': the fast reciprocal
// (within 2 ulp). The binning's corner keys, the composite, the replay and the backward re-merge all
// take it from here, so that their decisions agree bit for bit; against the FP64 oracle its error is
// far inside the decision margins (2e-5 relative).
__device__ __forceinline__ float rec_rcp(float A) { return __fdividef(1.f, A); }

// The exact hit decision (alpha >= 1/255 and t* > near) for a pixel whose pre-test passed.
// Returns t*' and alpha.
__device__ __forceinline__ bool rec_hit(const RecEval &e, const float4 &r0, const float4 &r2, float dnorm,
                                        float near_plane, float &tp, float &a) {
    const float rA = rec_rcp(e.A);
    const float m = __fmul_rn(e.N, rA);
    a = fminf(kAlphaMax, __fmul_rn(r0.w, __expf(-0.5f * m)));
    tp = __fmul_rn(-rec_od(r2, e.dx, e.dy), rA);
    return a >= kAlphaMin && __fmul_rn(tp, dnorm) > near_plane;
}

}  // namespace sof
