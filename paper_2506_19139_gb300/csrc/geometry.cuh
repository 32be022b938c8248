// Per-(Gaussian, view) geometry shared by the forward preprocess and its backward.
//
// The paper evaluates each Gaussian along a ray in Gaussian space, o_g = S^-1 R^T (o - mu),
// d_g = S^-1 R^T d (Sec. 3.1 "Gaussian Opacity Fields"; the rotation enters transposed because
// R maps local to world, Sigma = R S S^T R^T). Evaluating m = C - B^2/4A directly in FP32 cancels
// catastrophically for small Gaussians far from the camera (C ~ 1e5 in the tiny configuration),
// so the record instead holds the affine pixel-plane expansion of the cross product o_g x d_g
// (|o_g x d_g|^2 / |d_g|^2 = C - B^2/4A, Lagrange's identity) around an anchor pixel:
//   o_g x d_g(pixel) = C0 + dx P + dy Q,  P = o_g x a, Q = o_g x b, C0 = o_g x d_g(anchor),
// with a, b the Gaussian-space images of one pixel step in x and y. P, Q and C0 are computed
// with the cofactor identity (M u) x (M v) = det(M) M^-T (u x v) from world-space cross products
// whose only cancelling one (C0) is formed in FP64 from the FP64 camera-space mean, so every
// record coefficient is accurate relative to its own size.
#pragma once

#include <math.h>

#include "sof_internal.cuh"

namespace sof {

struct F3 {
    float x, y, z;
};
__device__ __forceinline__ F3 f3(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot3(F3 a, F3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ F3 cross3(F3 a, F3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float norm3(F3 a) { return sqrtf(dot3(a, a)); }

// Quaternion (w,x,y,z) -> rotation, normalised; R[i][j] row-major, columns = principal axes.
__device__ __forceinline__ void quat_to_rotation(float4 q, float R[3][3], float *qn_out) {
    float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
    if (qn_out) { qn_out[0] = w; qn_out[1] = x; qn_out[2] = y; qn_out[3] = z; }
    R[0][0] = 1.f - 2.f * (y * y + z * z); R[0][1] = 2.f * (x * y - w * z); R[0][2] = 2.f * (x * z + w * y);
    R[1][0] = 2.f * (x * y + w * z); R[1][1] = 1.f - 2.f * (x * x + z * z); R[1][2] = 2.f * (y * z - w * x);
    R[2][0] = 2.f * (x * z - w * y); R[2][1] = 2.f * (y * z + w * x); R[2][2] = 1.f - 2.f * (x * x + y * y);
}

// Real spherical harmonics, degree <= 3, 3DGS ordering and signs. Constants are the closed-form
// normalisations: 1/(2 sqrt(pi)), sqrt(3/(4 pi)), sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4,
// sqrt(35/(2 pi))/4, sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
__device__ __forceinline__ int sh_eval_basis(int degree, F3 d, float *Y) {
    const float k0 = 0.28209479177387814f, k1 = 0.4886025119029199f;
    const float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.5462742152960396f;
    const float k3a = 0.5900435899266435f, k3b = 2.890611442640554f, k3c = 0.4570457994644658f;
    const float k3d = 0.3731763325901154f, k3e = 1.445305721320277f;
    Y[0] = k0;
    if (degree < 1) return 1;
    float x = d.x, y = d.y, z = d.z;
    Y[1] = -k1 * y; Y[2] = k1 * z; Y[3] = -k1 * x;
    if (degree < 2) return 4;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = k2a * x * y; Y[5] = -k2a * y * z; Y[6] = k2b * (2.f * zz - xx - yy);
    Y[7] = -k2a * x * z; Y[8] = k2c * (xx - yy);
    if (degree < 3) return 9;
    Y[9] = -k3a * y * (3.f * xx - yy);
    Y[10] = k3b * x * y * z;
    Y[11] = -k3c * y * (4.f * zz - xx - yy);
    Y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -k3c * x * (4.f * zz - xx - yy);
    Y[14] = k3e * z * (xx - yy);
    Y[15] = -k3a * x * (xx - 3.f * yy);
    return 16;
}

// d Y_k / d dir (un-normalised partials with respect to x, y, z), degree <= 3.
__device__ __forceinline__ void sh_eval_basis_grad(int degree, F3 d, F3 *dY) {
    const float k1 = 0.4886025119029199f;
    const float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.5462742152960396f;
    const float k3a = 0.5900435899266435f, k3b = 2.890611442640554f, k3c = 0.4570457994644658f;
    const float k3d = 0.3731763325901154f, k3e = 1.445305721320277f;
    float x = d.x, y = d.y, z = d.z;
    dY[0] = f3(0.f, 0.f, 0.f);
    if (degree < 1) return;
    dY[1] = f3(0.f, -k1, 0.f); dY[2] = f3(0.f, 0.f, k1); dY[3] = f3(-k1, 0.f, 0.f);
    if (degree < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    dY[4] = f3(k2a * y, k2a * x, 0.f);
    dY[5] = f3(0.f, -k2a * z, -k2a * y);
    dY[6] = f3(-2.f * k2b * x, -2.f * k2b * y, 4.f * k2b * z);
    dY[7] = f3(-k2a * z, 0.f, -k2a * x);
    dY[8] = f3(2.f * k2c * x, -2.f * k2c * y, 0.f);
    if (degree < 3) return;
    dY[9] = f3(-k3a * 6.f * x * y, -k3a * (3.f * xx - 3.f * yy), 0.f);
    dY[10] = f3(k3b * y * z, k3b * x * z, k3b * x * y);
    dY[11] = f3(k3c * 2.f * x * y, -k3c * (4.f * zz - xx - 3.f * yy), -k3c * 8.f * y * z);
    dY[12] = f3(-k3d * 6.f * x * z, -k3d * 6.f * y * z, k3d * (6.f * zz - 3.f * xx - 3.f * yy));
    dY[13] = f3(-k3c * (4.f * zz - 3.f * xx - yy), k3c * 2.f * x * y, -k3c * 8.f * x * z);
    dY[14] = f3(k3e * 2.f * x * z, -k3e * 2.f * y * z, k3e * (xx - yy));
    dY[15] = f3(-k3a * (3.f * xx - 3.f * yy), k3a * 6.f * x * y, 0.f);
}

// Everything the record of one (Gaussian, view) is built from.
struct GaussView {
    bool visible;
    float o, E2, s[3], R[3][3];     // opacity, cut-off^2, scales, rotation (local -> world)
    float M[3][3];                  // S^-1 R^T (world -> Gaussian space)
    double xc[3];                   // camera-space mean, FP64
    F3 w;                           // mu - c (world), FP32
    F3 og, dga, a, b;               // Gaussian-space o_g, d_g(anchor), pixel steps
    F3 P, Q, C0, e1, e2;            // cross-product expansion and plane basis
    float p1, q1, q2, c1, c2;       // expansion in the basis
    float ia, ja;                   // anchor pixel
    float delta_x, delta_y;         // anchor centre minus projected mean (pixels)
    bool proj_ok;                   // anchor from a valid projection of the mean
    float dist;                     // |mu - c|
    float zmin, zmax;               // camera-z extent of the E-ellipsoid
    float t_lo;                     // Euclidean lower bound on t* of any hit
    float sxx, syy, szz, sxz, syz;  // camera-space covariance entries
    int kmin;                       // smallest-scale axis
    int px0, px1, py0, py1;         // inclusive pixel-index bounding box of the silhouette
    float rho2;                     // squared silhouette cone radius with the pre-test slack (< 0: inside)
};

constexpr float kPreTest = 1.0f + 1e-4f;  // relative slack on E^2 for the conservative pre-tests

// Conservative screen rectangle of the silhouette of the E-ellipsoid (inclusive pixel-index
// bounding box, padded by one pixel plus a relative margin) and the squared radius of the
// silhouette cone in Gaussian space. Returns false if the rectangle misses the image.
__device__ __forceinline__ bool screen_rect(GaussView &G, const DevCam &cam) {
    const float E = sqrtf(G.E2);
    const float xc = (float)G.xc[0], yc = (float)G.xc[1], zc = (float)G.xc[2];
    float ulo, uhi, vlo, vhi;
    const float C = dot3(G.og, G.og);
    const bool inside = C <= G.E2 * kPreTest;
    G.rho2 = inside ? -1.f : G.E2 * kPreTest / (C - G.E2 * kPreTest);
    if (inside) {
        ulo = vlo = -1e30f;
        uhi = vhi = 1e30f;
    } else if (G.zmin > cam.zclip) {
        // tangent planes through the camera centre: exact extent of the silhouette
        const float aq = zc * zc - G.E2 * G.szz;
        const float bx = xc * zc - G.E2 * G.sxz, by = yc * zc - G.E2 * G.syz;
        const float dx = G.E2 * ((zc * zc * G.sxx - 2.f * xc * zc * G.sxz + xc * xc * G.szz) -
                                 G.E2 * (G.sxx * G.szz - G.sxz * G.sxz));
        const float dy = G.E2 * ((zc * zc * G.syy - 2.f * yc * zc * G.syz + yc * yc * G.szz) -
                                 G.E2 * (G.syy * G.szz - G.syz * G.syz));
        const float sdx = sqrtf(fmaxf(dx, 0.f)), sdy = sqrtf(fmaxf(dy, 0.f));
        ulo = (bx - sdx) / aq; uhi = (bx + sdx) / aq;
        vlo = (by - sdy) / aq; vhi = (by + sdy) / aq;
    } else {
        // straddles the clip depth: project the camera-space bounding box clipped at zclip
        const float zl = fmaxf(G.zmin, cam.zclip), zh = G.zmax;
        const float ex = E * sqrtf(G.sxx), ey = E * sqrtf(G.syy);
        const float xl = xc - ex, xh = xc + ex, yl = yc - ey, yh = yc + ey;
        ulo = fminf(fminf(xl / zl, xl / zh), fminf(xh / zl, xh / zh));
        uhi = fmaxf(fmaxf(xl / zl, xl / zh), fmaxf(xh / zl, xh / zh));
        vlo = fminf(fminf(yl / zl, yl / zh), fminf(yh / zl, yh / zh));
        vhi = fmaxf(fmaxf(yl / zl, yl / zh), fmaxf(yh / zl, yh / zh));
    }
    // to pixel coordinates, inflated by one pixel plus a relative margin
    auto clampf = [](float x) { return fminf(fmaxf(x, -1e9f), 1e9f); };
    const float Xlo = clampf(cam.cx + cam.fx * ulo), Xhi = clampf(cam.cx + cam.fx * uhi);
    const float Ylo = clampf(cam.cy + cam.fy * vlo), Yhi = clampf(cam.cy + cam.fy * vhi);
    const float padx = 1.f + 1e-5f * (fabsf(Xlo) + fabsf(Xhi)), pady = 1.f + 1e-5f * (fabsf(Ylo) + fabsf(Yhi));
    G.px0 = (int)fmaxf(ceilf(Xlo - padx - 0.5f), 0.f);
    G.px1 = (int)fminf(floorf(Xhi + padx - 0.5f), (float)(cam.W - 1));
    G.py0 = (int)fmaxf(ceilf(Ylo - pady - 0.5f), 0.f);
    G.py1 = (int)fminf(floorf(Yhi + pady - 0.5f), (float)(cam.H - 1));
    return G.px0 <= G.px1 && G.py0 <= G.py1;
}

// Builds the geometry of Gaussian g in camera `cam`. Returns false (visible=false) if the
// Gaussian is dead (o <= 1/255), non-finite, cannot produce a hit with t* > near_plane, or has a
// silhouette rectangle outside the image (tested before the record's expansion is built).
// With cull_only, returns after the culling tests (everything up to the screen rectangle): the
// record's expansion and the FP64 work it needs are left out.
__device__ __forceinline__ bool gauss_view(const SceneDev &sc, long long g, const DevCam &cam,
                                           float near_plane, GaussView &G, bool *nonfinite,
                                           bool cull_only = false) {
    G.visible = false;
    const float *mp = sc.means + 3 * g;
    const float *lp = sc.log_scales + 3 * g;
    float4 q = reinterpret_cast<const float4 *>(sc.quats)[g];
    float mu[3] = {mp[0], mp[1], mp[2]};
    float ls[3] = {lp[0], lp[1], lp[2]};
    float logit = sc.logits[g];
    bool fin = isfinite(mu[0]) && isfinite(mu[1]) && isfinite(mu[2]) && isfinite(ls[0]) &&
               isfinite(ls[1]) && isfinite(ls[2]) && isfinite(q.x) && isfinite(q.y) && isfinite(q.z) &&
               isfinite(q.w) && isfinite(logit) && (q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w) > 0.f;
    if (nonfinite) *nonfinite = !fin;
    if (!fin) return false;
    G.o = 1.f / (1.f + expf(-logit));
    if (!(G.o > kAlphaMin)) return false;  // dead Gaussians never reach 1/255 (Sec. 3.4)
    G.E2 = 2.f * logf(255.f * G.o);        // Eq. 3, squared
    float E = sqrtf(G.E2);
    for (int k = 0; k < 3; ++k) G.s[k] = expf(ls[k]);
    quat_to_rotation(q, G.R, nullptr);
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) G.M[k][j] = G.R[j][k] / G.s[k];
    G.kmin = 0;
    if (G.s[1] < G.s[G.kmin]) G.kmin = 1;
    if (G.s[2] < G.s[G.kmin]) G.kmin = 2;
    float smax = fmaxf(G.s[0], fmaxf(G.s[1], G.s[2]));

    // camera-space mean in FP64 (products of FP32 values are exact in FP64)
    for (int i = 0; i < 3; ++i)
        G.xc[i] = cam.R[3 * i] * (double)mu[0] + cam.R[3 * i + 1] * (double)mu[1] +
                  cam.R[3 * i + 2] * (double)mu[2] + cam.t[i];
    float xcf[3] = {(float)G.xc[0], (float)G.xc[1], (float)G.xc[2]};
    // a float square root of the FP64 sum: within an ulp of the rounded FP64 root, at FP32 cost
    G.dist = sqrtf((float)(G.xc[0] * G.xc[0] + G.xc[1] * G.xc[1] + G.xc[2] * G.xc[2]));
    if (G.dist + E * smax < near_plane) return false;  // whole ellipsoid inside the near sphere

    // camera-space covariance: V_k = R_c R[:,k] s_k
    float Vc[3][3];
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i)
            Vc[k][i] = (cam.Rf[3 * i] * G.R[0][k] + cam.Rf[3 * i + 1] * G.R[1][k] + cam.Rf[3 * i + 2] * G.R[2][k]) * G.s[k];
    G.sxx = G.syy = G.szz = G.sxz = G.syz = 0.f;
    for (int k = 0; k < 3; ++k) {
        G.sxx = fmaf(Vc[k][0], Vc[k][0], G.sxx);
        G.syy = fmaf(Vc[k][1], Vc[k][1], G.syy);
        G.szz = fmaf(Vc[k][2], Vc[k][2], G.szz);
        G.sxz = fmaf(Vc[k][0], Vc[k][2], G.sxz);
        G.syz = fmaf(Vc[k][1], Vc[k][2], G.syz);
    }
    float sz = sqrtf(G.szz);
    G.zmin = xcf[2] - E * sz;
    G.zmax = xcf[2] + E * sz;
    if (G.zmax <= cam.zclip) return false;  // no in-image ray reaches it beyond the near plane

    // world vector mu - c = R_c^T xc, and o_g = S^-1 R^T (c - mu)
    G.w = f3(cam.Rf[0] * xcf[0] + cam.Rf[3] * xcf[1] + cam.Rf[6] * xcf[2],
             cam.Rf[1] * xcf[0] + cam.Rf[4] * xcf[1] + cam.Rf[7] * xcf[2],
             cam.Rf[2] * xcf[0] + cam.Rf[5] * xcf[1] + cam.Rf[8] * xcf[2]);
    auto Mv = [&](F3 u) {
        return f3(G.M[0][0] * u.x + G.M[0][1] * u.y + G.M[0][2] * u.z,
                  G.M[1][0] * u.x + G.M[1][1] * u.y + G.M[1][2] * u.z,
                  G.M[2][0] * u.x + G.M[2][1] * u.y + G.M[2][2] * u.z);
    };
    G.og = -1.f * Mv(G.w);
    {
        // Every peak point c + t* d lies on the ellipsoid (p - c)^T Sigma^-1 (p - mu) = 0, centred at
        // (c + mu) / 2 with Mahalanobis radius sqrt(C) / 2, so t* <= (|mu - c| + s_max sqrt(C)) / 2.
        // A Gaussian whose bound stays below the near plane can never be hit (Sec. 3.3 near test):
        // typically one that contains the camera and would otherwise cover every tile.
        const float C = dot3(G.og, G.og);
        if (0.5f * (G.dist + smax * sqrtf(C)) * 1.001f < near_plane) return false;
    }
    if (!screen_rect(G, cam)) return false;
    if (cull_only) return true;

    // anchor pixel: the pixel containing the projected mean, else the image centre
    double Xm = 0.0, Ym = 0.0;
    G.proj_ok = false;
    if (G.xc[2] > 1e-6 * (double)G.dist) {
        const double iz = recip_fp64(G.xc[2]);
        Xm = (double)cam.fx * (G.xc[0] * iz) + (double)cam.cx;
        Ym = (double)cam.fy * (G.xc[1] * iz) + (double)cam.cy;
        G.proj_ok = fabs(Xm) < 1048576.0 && fabs(Ym) < 1048576.0;
    }
    if (G.proj_ok) {
        G.ia = (float)floor(Xm);
        G.ja = (float)floor(Ym);
        G.delta_x = (float)((double)G.ia + 0.5 - Xm);
        G.delta_y = (float)((double)G.ja + 0.5 - Ym);
    } else {
        G.ia = floorf(cam.cx);
        G.ja = floorf(cam.cy);
        G.delta_x = G.delta_y = 0.f;
    }
    double ua = ((double)G.ia + 0.5 - (double)cam.cx) * cam.rfx;
    double va = ((double)G.ja + 0.5 - (double)cam.cy) * cam.rfy;

    // world directions of the anchor ray and of one pixel step (rows of R_c)
    F3 r0 = f3(cam.Rf[0], cam.Rf[1], cam.Rf[2]), r1 = f3(cam.Rf[3], cam.Rf[4], cam.Rf[5]);
    F3 r2 = f3(cam.Rf[6], cam.Rf[7], cam.Rf[8]);
    float rfx = 1.f / cam.fx, rfy = 1.f / cam.fy;
    F3 wx = rfx * r0, wy = rfy * r1;
    F3 wa = (float)ua * r0 + (float)va * r1 + r2;
    G.dga = Mv(wa);
    G.a = Mv(wx);
    G.b = Mv(wy);
    // cofactor of M: row k = R[:,k]^T / (s_{k+1} s_{k+2})
    float cf[3] = {1.f / (G.s[1] * G.s[2]), 1.f / (G.s[0] * G.s[2]), 1.f / (G.s[0] * G.s[1])};
    auto Cof = [&](F3 u) {
        return f3(cf[0] * (G.R[0][0] * u.x + G.R[1][0] * u.y + G.R[2][0] * u.z),
                  cf[1] * (G.R[0][1] * u.x + G.R[1][1] * u.y + G.R[2][1] * u.z),
                  cf[2] * (G.R[0][2] * u.x + G.R[1][2] * u.y + G.R[2][2] * u.z));
    };
    // (c - mu) x w = -R_c^T (xc x w_cam); for w_cam = (1/fx,0,0), (0,1/fy,0), (ua,va,1)
    auto rotT = [&](double cx_, double cy_, double cz_) {
        float X = (float)cx_, Y = (float)cy_, Z = (float)cz_;
        return -1.f * (X * r0 + Y * r1 + Z * r2);
    };
    G.P = Cof(rotT(0.0, G.xc[2] * cam.rfx, -G.xc[1] * cam.rfx));
    G.Q = Cof(rotT(-G.xc[2] * cam.rfy, 0.0, G.xc[0] * cam.rfy));
    G.C0 = Cof(rotT(G.xc[1] - G.xc[2] * va, G.xc[2] * ua - G.xc[0], G.xc[0] * va - G.xc[1] * ua));

    // orthonormal basis of the plane normal to o_g, e1 along P
    float on = norm3(G.og);
    F3 oh = on > 0.f ? (1.f / on) * G.og : f3(0.f, 0.f, 1.f);
    G.p1 = norm3(G.P);
    float qn = norm3(G.Q);
    if (G.p1 > 1e-30f && G.p1 > 1e-12f * qn) {
        G.e1 = (1.f / G.p1) * G.P;
    } else {
        F3 t = fabsf(oh.x) < 0.9f ? f3(1.f, 0.f, 0.f) : f3(0.f, 1.f, 0.f);
        F3 e = cross3(oh, t);
        G.e1 = (1.f / norm3(e)) * e;
        G.p1 = 0.f;
    }
    G.e2 = cross3(oh, G.e1);
    G.q1 = dot3(G.Q, G.e1);
    if (G.p1 > 0.f) {
        // P x Q = (o_g . (a x b)) o_g and o_g . (a x b) = -z_mu / (s0 s1 s2 fx fy)
        G.q2 = (float)(-G.xc[2]) * on * rfx * rfy / (G.s[0] * G.s[1] * G.s[2] * G.p1);
    } else {
        G.q2 = dot3(G.Q, G.e2);
    }
    G.c1 = dot3(G.C0, G.e1);
    G.c2 = dot3(G.C0, G.e2);

    // Euclidean lower bound on t* of any hit: the peak lies inside the E-ellipsoid, whose
    // distance along the unit direction to the mean is at least |mu-c| - E sigma_view.
    F3 dh = (1.f / fmaxf(G.dist, 1e-30f)) * G.w;
    float sv2 = 0.f;
    for (int k = 0; k < 3; ++k) {
        float pr = G.R[0][k] * dh.x + G.R[1][k] * dh.y + G.R[2][k] * dh.z;
        sv2 = fmaf(G.s[k] * G.s[k], pr * pr, sv2);
    }
    G.t_lo = fmaxf(near_plane, G.dist - E * sqrtf(sv2));
    G.visible = true;
    return true;
}

}  // namespace sof
