// Backward of the per-(Gaussian, view) preprocessing: chains the per-record gradients written by
// the backward composite to means, log-scales, quaternions, opacity logits and SH coefficients.
// One thread per Gaussian loops over the views, so no atomics are needed; gradients are added
// (+=) to the caller's buffers.
//
// Record gradient layout (22 used floats of 24):
//   [0,1]   dL/dC0 in the plane basis (e1, e2)       [2,3] dL/dP    [4,5] dL/dQ
//   [6..11] dL/d(a00, ax, ay, axx, axy, ayy)         [12..14] dL/d(od0, odx, ody)
//   [15]    dL/do                                    [16..18] dL/drgb   [19..21] dL/dnormal
// The cross-product terms are basis-free: N = |C0 + dx P + dy Q|^2 with C0, P, Q normal to o_g,
// so dL/dC0 (3D) = e1 g0 + e2 g1 and likewise for P and Q.
#include <math.h>

#include "geometry.cuh"
#include "sof_internal.cuh"

namespace sof {
namespace {

__global__ void __launch_bounds__(128) k_preprocess_bwd(SceneDev sc, const CamSet *__restrict__ cams, int n_views,
                                                        float near_plane, const int *__restrict__ vflag,
                                                        const int *__restrict__ vis_pos, int vis_cap,
                                                        const float4 *__restrict__ rgrad, sof_scene_grad grad) {
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= sc.n) return;
    const long long n = sc.n;
    const int K = (sc.sh_degree + 1) * (sc.sh_degree + 1);
    float gmu[3] = {0.f, 0.f, 0.f}, glogs[3] = {0.f, 0.f, 0.f}, gR[3][3] = {{0.f}}, glogit = 0.f;
    float4 qraw = reinterpret_cast<const float4 *>(sc.quats)[g];
    bool any = false;
    for (int v = 0; v < n_views; ++v) {
        long long rec = (long long)v * n + g;
        if (!vflag[rec]) continue;  // no tile, no hit, no gradient
        const int k = vis_pos[rec];
        if (k >= vis_cap) continue;
        const float4 *gp = rgrad + (size_t)k * kGradF4;
        float gr[24];
        for (int k = 0; k < 6; ++k) {
            float4 x = gp[k];
            gr[4 * k] = x.x; gr[4 * k + 1] = x.y; gr[4 * k + 2] = x.z; gr[4 * k + 3] = x.w;
        }
        bool nz = false;
        for (int k = 0; k < 22; ++k) nz |= (gr[k] != 0.f);
        if (!nz) continue;
        any = true;
        const DevCam &cam = cams->cam[v];
        GaussView G;
        if (!gauss_view(sc, g, cam, near_plane, G, nullptr)) continue;

        F3 gC0 = gr[0] * G.e1 + gr[1] * G.e2;
        F3 gP = gr[2] * G.e1 + gr[3] * G.e2;
        F3 gQ = gr[4] * G.e1 + gr[5] * G.e2;
        float gA0 = gr[6], gAx = gr[7], gAy = gr[8], gAxx = gr[9], gAxy = gr[10], gAyy = gr[11];
        float god0 = gr[12], godx = gr[13], gody = gr[14], go = gr[15];
        // to the Gaussian-space vectors o_g, d_g(anchor), a, b
        F3 g_og = cross3(G.dga, gC0) + cross3(G.a, gP) + cross3(G.b, gQ) + god0 * G.dga + godx * G.a + gody * G.b;
        F3 g_dga = cross3(gC0, G.og) + (2.f * gA0) * G.dga + (2.f * gAx) * G.a + (2.f * gAy) * G.b + god0 * G.og;
        F3 g_a = cross3(gP, G.og) + (2.f * gAx) * G.dga + (2.f * gAxx) * G.a + (2.f * gAxy) * G.b + godx * G.og;
        F3 g_b = cross3(gQ, G.og) + (2.f * gAy) * G.dga + (2.f * gAxy) * G.a + (2.f * gAyy) * G.b + gody * G.og;
        // o_g = -M w, d_g(anchor) = M w_a, a = M w_x, b = M w_y with M = S^-1 R^T
        F3 r0 = f3(cam.Rf[0], cam.Rf[1], cam.Rf[2]), r1 = f3(cam.Rf[3], cam.Rf[4], cam.Rf[5]);
        F3 r2 = f3(cam.Rf[6], cam.Rf[7], cam.Rf[8]);
        double ua = ((double)G.ia + 0.5 - (double)cam.cx) * cam.rfx;
        double va = ((double)G.ja + 0.5 - (double)cam.cy) * cam.rfy;
        F3 wx = (1.f / cam.fx) * r0, wy = (1.f / cam.fy) * r1;
        F3 wa = (float)ua * r0 + (float)va * r1 + r2;
        float gog[3] = {g_og.x, g_og.y, g_og.z}, gdg[3] = {g_dga.x, g_dga.y, g_dga.z};
        float ga[3] = {g_a.x, g_a.y, g_a.z}, gb[3] = {g_b.x, g_b.y, g_b.z};
        float w[3] = {G.w.x, G.w.y, G.w.z}, wav[3] = {wa.x, wa.y, wa.z};
        float wxv[3] = {wx.x, wx.y, wx.z}, wyv[3] = {wy.x, wy.y, wy.z};
        for (int k = 0; k < 3; ++k) {
            float gl = 0.f;
            for (int j = 0; j < 3; ++j) {
                float gM = -gog[k] * w[j] + gdg[k] * wav[j] + ga[k] * wxv[j] + gb[k] * wyv[j];
                gR[j][k] += gM / G.s[k];
                gl -= gM * G.M[k][j];
            }
            glogs[k] += gl;
        }
        for (int j = 0; j < 3; ++j) {
            float s = 0.f;
            for (int k = 0; k < 3; ++k) s += G.M[k][j] * gog[k];
            gmu[j] -= s;  // w = mu - c
        }
        // normal = +-R[:, kmin] facing the camera
        F3 nrm = f3(G.R[0][G.kmin], G.R[1][G.kmin], G.R[2][G.kmin]);
        float sgn = dot3(nrm, G.w) > 0.f ? -1.f : 1.f;
        gR[0][G.kmin] += sgn * gr[19];
        gR[1][G.kmin] += sgn * gr[20];
        gR[2][G.kmin] += sgn * gr[21];
        // opacity
        glogit += go * G.o * (1.f - G.o);
        // colour: rgb = max(0, sum_k Y_k(dir) f_k + 0.5), dir = (mu - c)/|mu - c|
        if (gr[16] != 0.f || gr[17] != 0.f || gr[18] != 0.f) {
            float inv = 1.f / fmaxf(G.dist, 1e-30f);
            F3 dir = inv * G.w;
            float Y[16];
            F3 dY[16];
            sh_eval_basis(sc.sh_degree, dir, Y);
            sh_eval_basis_grad(sc.sh_degree, dir, dY);
            const float *shp = sc.sh + (size_t)g * K * 3;
            float *gsh = grad.d_sh ? grad.d_sh + (size_t)g * K * 3 : nullptr;
            F3 gdir = f3(0.f, 0.f, 0.f);
            for (int ch = 0; ch < 3; ++ch) {
                float col = 0.5f;
                for (int k = 0; k < K; ++k) col = fmaf(Y[k], shp[k * 3 + ch], col);
                float gc = gr[16 + ch];
                if (!(col > 0.f) || gc == 0.f) continue;
                for (int k = 0; k < K; ++k) {
                    if (gsh) gsh[k * 3 + ch] += Y[k] * gc;
                    gdir = gdir + (gc * shp[k * 3 + ch]) * dY[k];
                }
            }
            float pd = dot3(gdir, dir);
            F3 gw = inv * (gdir - pd * dir);
            gmu[0] += gw.x; gmu[1] += gw.y; gmu[2] += gw.z;
        }
    }
    if (!any) return;
    // rotation -> normalised quaternion -> raw quaternion
    float inv = rsqrtf(qraw.x * qraw.x + qraw.y * qraw.y + qraw.z * qraw.z + qraw.w * qraw.w);
    float qw = qraw.x * inv, qx = qraw.y * inv, qy = qraw.z * inv, qz = qraw.w * inv;
    float gw_ = 2.f * (-qz * gR[0][1] + qy * gR[0][2] + qz * gR[1][0] - qx * gR[1][2] - qy * gR[2][0] + qx * gR[2][1]);
    float gx_ = 2.f * (qy * gR[0][1] + qz * gR[0][2] + qy * gR[1][0] - 2.f * qx * gR[1][1] - qw * gR[1][2] +
                       qz * gR[2][0] + qw * gR[2][1] - 2.f * qx * gR[2][2]);
    float gy_ = 2.f * (-2.f * qy * gR[0][0] + qx * gR[0][1] + qw * gR[0][2] + qx * gR[1][0] + qz * gR[1][2] -
                       qw * gR[2][0] + qz * gR[2][1] - 2.f * qy * gR[2][2]);
    float gz_ = 2.f * (-2.f * qz * gR[0][0] - qw * gR[0][1] + qx * gR[0][2] + qw * gR[1][0] - 2.f * qz * gR[1][1] +
                       qy * gR[1][2] + qx * gR[2][0] + qy * gR[2][1]);
    float pr = gw_ * qw + gx_ * qx + gy_ * qy + gz_ * qz;
    if (grad.d_quats) {
        float *gq = grad.d_quats + 4 * g;
        gq[0] += (gw_ - pr * qw) * inv;
        gq[1] += (gx_ - pr * qx) * inv;
        gq[2] += (gy_ - pr * qy) * inv;
        gq[3] += (gz_ - pr * qz) * inv;
    }
    if (grad.d_means)
        for (int i = 0; i < 3; ++i) grad.d_means[3 * g + i] += gmu[i];
    if (grad.d_log_scales)
        for (int i = 0; i < 3; ++i) grad.d_log_scales[3 * g + i] += glogs[i];
    if (grad.d_opacity_logits) grad.d_opacity_logits[g] += glogit;
}

// Zero the gradient copies of the visible records (compacted: the first n_vis slots; grid-stride).
__global__ void k_grad_copies_zero(float4 *__restrict__ copies, const int *__restrict__ n_vis_dev, long long vis_cap) {
    const long long n = min((long long)*n_vis_dev, vis_cap) * kGradCopies * kGradF4;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        copies[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Sum the kGradCopies gradient copies of each visible record into its gradient (one thread per
// (record, float4 field), grid-stride over the compacted records).
__global__ void k_grad_copies_reduce(const float4 *__restrict__ copies, const int *__restrict__ n_vis_dev,
                                     long long vis_cap, float4 *__restrict__ rgrad) {
    const long long n = min((long long)*n_vis_dev, vis_cap) * kGradF4;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long k = i / kGradF4;
        const int g = (int)(i - k * kGradF4);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < kGradCopies; ++c) {
            const float4 v = copies[(k * kGradCopies + c) * kGradF4 + g];
            acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
        }
        rgrad[i] = acc;
    }
}

}  // namespace

cudaError_t launch_grad_copies_zero(float4 *copies, const int *n_vis_dev, long long vis_cap, cudaStream_t s) {
    if (vis_cap <= 0) return cudaSuccess;
    note_launches(1);
    k_grad_copies_zero<<<device_sm_count() * 8, 256, 0, s>>>(copies, n_vis_dev, vis_cap);
    return cudaGetLastError();
}

cudaError_t launch_grad_copies_reduce(const float4 *copies, const int *n_vis_dev, long long vis_cap, float4 *rgrad,
                                      cudaStream_t s) {
    if (vis_cap <= 0) return cudaSuccess;
    note_launches(1);
    k_grad_copies_reduce<<<device_sm_count() * 8, 256, 0, s>>>(copies, n_vis_dev, vis_cap, rgrad);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(const SceneDev &sc, const CamSet *cams_dev, int n_views, float near_plane,
                                  const int *vflag, const int *vis_pos, int vis_cap, const float4 *rgrad,
                                  const sof_scene_grad &grad, cudaStream_t s) {
    if (sc.n == 0) return cudaSuccess;
    int threads = 128;
    long long blocks = (sc.n + threads - 1) / threads;
    note_launches(1);
    k_preprocess_bwd<<<(unsigned)blocks, threads, 0, s>>>(sc, cams_dev, n_views, near_plane, vflag, vis_pos, vis_cap,
                                                         rgrad, grad);
    return cudaGetLastError();
}

}  // namespace sof
