/*
 * sof_oracle.c -- plain FP64 CPU oracle for the Sorted Opacity Fields compositing core.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call this file: only
 * tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg use it, to check and time the
 * CUDA library. It shares no code, header, table or constant generator with the CUDA path.
 *
 * It computes, slowly and directly, what the method defines:
 *   - 3D Gaussians with covariance Sigma = R S S^T R^T (Sec. 3.1 "Preliminaries"),
 *   - the per-ray quadratic A t^2 + B t + C, its peak t* = -B/2A and the peak response
 *     G = exp(-1/2 (C - B^2/4A))  (Sec. 3.1 "Gaussian Opacity Fields", Eqs. 6-10),
 *   - front-to-back alpha blending in exact per-pixel t* order (Eq. 1, Sec. 3.1 "StopThePop"),
 *   - the opacity cut-off E = sqrt(2 ln(255 o)) (Eq. 3, Sec. 3.4 "Tighter Gaussian Bounding"),
 *   - the exact depth solving T_k (1 - o_k G(t)) = 0.5 on the crossing Gaussian
 *     (Sec. 3.2 "Exact Depth", App. A.3),
 *   - the opacity field O_N at points with t_eval = min(t*, t) and the min over views
 *     (Eqs. 11-12, App. A.2),
 *   - the distortion and extent loss channels over a pixel's composited hits (Sec. 3.3,
 *     App. C.1-C.2) and the opacity field at the exact-depth point of a pixel's ray (Sec. 3.3,
 *     L_opa).
 * Readings of silent or garbled passages (quaternion convention, SH convention, normal, stop
 * rule, no-crossing value, near test, the losses' NDC map) are the ones listed in the design notes
 * and are marked READING below.
 *
 * Pinning status: every function here is pinned by tests/test_oracle_pins.py against closed
 * forms, textbook geometry, brute force and invariants, and tests/test_oracle_mutations.py checks
 * that planted mistakes fail those pins. The paper prints no worked numeric example, so no value
 * here is pinned against a number printed in the paper. The normal channel follows the reading of
 * the paper's "normal as defined in GOF" (the axis of the smallest scale, facing the camera) and is
 * pinned against that reading only: parity unpinned against the paper's own definition, which it
 * does not give.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC sof_oracle.c -o libsof_oracle.so -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99

/* decision-margin flag bits (several correct results exist near a threshold) */
#define FLAG_ALPHA 1   /* an alpha within the margin of 1/255                         */
#define FLAG_TSTOP 2   /* a transmittance within the margin of the stop threshold      */
#define FLAG_NEAR 4    /* a t* within the margin of the near plane                     */
#define FLAG_ORDER 8   /* two composited hits with nearly equal t*                     */
#define FLAG_CROSS 16  /* transmittance within the margin of 0.5 at the crossing       */
#define FLAG_VIEW 32   /* query point on the edge of a view's frustum                  */
#define FLAG_OVERFLOW 64
#define FLAG_EXACT 128 /* exact depth ill-conditioned: FP32 inputs cannot resolve it to 1e-4  */
#define FLAG_UNRESOLVED 256 /* more decisions within their margins than the enumeration takes  */

typedef struct {
    double R[3][3]; /* world -> camera rotation */
    double t[3];
    double c[3];    /* camera centre in world coordinates, -R^T t */
    double fx, fy, cx, cy;
    int W, H;
} ocam;

typedef struct {
    double mu[3];
    double s[3];
    double Rg[3][3];   /* local -> world rotation; column k is principal axis k */
    double Sinv[3][3]; /* Sigma^{-1} = R diag(1/s^2) R^T */
    double o, E2, smax;
    int alive;
    double rgb[3];
    double n[3];
} ogauss;

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static void make_cam(const float *w2c, const float *intr, int W, int H, ocam *cam) {
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) cam->R[i][j] = (double)w2c[i * 4 + j];
        cam->t[i] = (double)w2c[i * 4 + 3];
    }
    for (int j = 0; j < 3; ++j) {
        double acc = 0.0;
        for (int i = 0; i < 3; ++i) acc -= cam->R[i][j] * cam->t[i];
        cam->c[j] = acc;
    }
    cam->fx = intr[0]; cam->fy = intr[1]; cam->cx = intr[2]; cam->cy = intr[3];
    cam->W = W; cam->H = H;
}

/* READING: quaternion stored (w,x,y,z), normalised, Hamilton convention, R maps local -> world
 * so that Sigma = R S S^T R^T (Sec. 3.1). */
static void quat_to_rot(const double q_in[4], double R[3][3]) {
    double nrm = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / nrm, x = q_in[1] / nrm, y = q_in[2] / nrm, z = q_in[3] / nrm;
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* READING: real spherical harmonics up to degree 3 in the ordering and sign convention of 3D
 * Gaussian Splatting; each constant is the textbook normalisation written as its closed form. */
int oracle_sh_basis(int degree, const double dir[3], double *Y) {
    const double pi = 3.14159265358979323846;
    double x = dir[0], y = dir[1], z = dir[2];
    Y[0] = 0.5 * sqrt(1.0 / pi);
    if (degree < 1) return 1;
    double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -c1 * y; Y[2] = c1 * z; Y[3] = -c1 * x;
    if (degree < 2) return 4;
    double xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 0.5 * sqrt(15.0 / pi) * x * y;
    Y[5] = -0.5 * sqrt(15.0 / pi) * y * z;
    Y[6] = 0.25 * sqrt(5.0 / pi) * (2.0 * zz - xx - yy);
    Y[7] = -0.5 * sqrt(15.0 / pi) * x * z;
    Y[8] = 0.25 * sqrt(15.0 / pi) * (xx - yy);
    if (degree < 3) return 9;
    Y[9] = -0.25 * sqrt(35.0 / (2.0 * pi)) * y * (3.0 * xx - yy);
    Y[10] = 0.5 * sqrt(105.0 / pi) * x * y * z;
    Y[11] = -0.25 * sqrt(21.0 / (2.0 * pi)) * y * (4.0 * zz - xx - yy);
    Y[12] = 0.25 * sqrt(7.0 / pi) * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = -0.25 * sqrt(21.0 / (2.0 * pi)) * x * (4.0 * zz - xx - yy);
    Y[14] = 0.25 * sqrt(105.0 / pi) * z * (xx - yy);
    Y[15] = -0.25 * sqrt(35.0 / (2.0 * pi)) * x * (xx - 3.0 * yy);
    return 16;
}

/* Per-Gaussian quantities that depend only on the Gaussian and the camera centre, from FP64
 * parameters (sh_row: K*3 coefficients of this Gaussian, or NULL for no colour). */
static void prep_gauss_d(const double mu[3], const double ls[3], const double q[4], double logit,
                         const double *sh_row, int sh_degree, const ocam *cam, ogauss *G) {
    int K = (sh_degree + 1) * (sh_degree + 1);
    for (int i = 0; i < 3; ++i) {
        G->mu[i] = mu[i];
        G->s[i] = exp(ls[i]);
    }
    quat_to_rot(q, G->Rg);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += G->Rg[i][k] * G->Rg[j][k] / (G->s[k] * G->s[k]);
            G->Sinv[i][j] = acc;
        }
    G->o = 1.0 / (1.0 + exp(-logit));
    G->alive = G->o > ALPHA_MIN;                       /* dead Gaussians never render (Sec. 3.4) */
    G->E2 = G->alive ? 2.0 * log(255.0 * G->o) : 0.0;  /* Eq. 3, squared */
    G->smax = fmax(G->s[0], fmax(G->s[1], G->s[2]));
    /* colour from SH along the view direction mean - camera centre (READING, 3DGS convention) */
    double dir[3], nrm = 0.0;
    for (int i = 0; i < 3; ++i) { dir[i] = G->mu[i] - cam->c[i]; nrm += dir[i] * dir[i]; }
    nrm = sqrt(nrm);
    for (int i = 0; i < 3; ++i) dir[i] /= nrm;
    double Y[16];
    oracle_sh_basis(sh_degree, dir, Y);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        if (sh_row)
            for (int k = 0; k < K; ++k) acc += Y[k] * sh_row[k * 3 + ch];
        G->rgb[ch] = acc > 0.0 ? acc : 0.0;
    }
    /* READING: Gaussian normal = principal axis of the smallest scale (lowest index on ties),
     * oriented towards the camera. */
    int kmin = 0;
    for (int k = 1; k < 3; ++k) if (G->s[k] < G->s[kmin]) kmin = k;
    double dotv = 0.0;
    for (int i = 0; i < 3; ++i) { G->n[i] = G->Rg[i][kmin]; dotv += G->n[i] * (G->mu[i] - cam->c[i]); }
    if (dotv > 0.0) for (int i = 0; i < 3; ++i) G->n[i] = -G->n[i];
}

/* The same from FP32 parameter arrays (every FP32 value is exact in FP64). */
static void prep_gauss(int64_t g, const float *means, const float *log_scales, const float *quats,
                       const float *logits, const float *sh, int sh_degree, const ocam *cam,
                       ogauss *G) {
    int K = (sh_degree + 1) * (sh_degree + 1);
    double mu[3], ls[3], q[4], shd[48];
    for (int i = 0; i < 3; ++i) { mu[i] = means[g * 3 + i]; ls[i] = log_scales[g * 3 + i]; }
    for (int i = 0; i < 4; ++i) q[i] = quats[g * 4 + i];
    if (sh)
        for (int k = 0; k < K * 3; ++k) shd[k] = sh[g * K * 3 + k];
    prep_gauss_d(mu, ls, q, (double)logits[g], sh ? shd : NULL, sh_degree, cam, G);
}

static void pixel_dir(const ocam *cam, int px, int py, double d[3]) {
    double u = ((double)px + 0.5 - cam->cx) / cam->fx;
    double v = ((double)py + 0.5 - cam->cy) / cam->fy;
    double nrm = 0.0;
    for (int j = 0; j < 3; ++j) {
        d[j] = cam->R[0][j] * u + cam->R[1][j] * v + cam->R[2][j];
        nrm += d[j] * d[j];
    }
    nrm = sqrt(nrm);
    for (int j = 0; j < 3; ++j) d[j] /= nrm;
}

/* The per-ray quadratic of Eq. 7: A = d^T Sigma^-1 d, B = 2 d^T Sigma^-1 (c - mu),
 * C = (c-mu)^T Sigma^-1 (c-mu), written in world space (equal to d_g^T d_g etc. of Eq. 4-5). */
static void ray_quadratic(const ogauss *G, const double c[3], const double d[3],
                          double *A, double *B, double *C) {
    double w[3], Sd[3], Sw[3];
    for (int i = 0; i < 3; ++i) w[i] = c[i] - G->mu[i];
    for (int i = 0; i < 3; ++i) {
        Sd[i] = G->Sinv[i][0] * d[0] + G->Sinv[i][1] * d[1] + G->Sinv[i][2] * d[2];
        Sw[i] = G->Sinv[i][0] * w[0] + G->Sinv[i][1] * w[1] + G->Sinv[i][2] * w[2];
    }
    *A = d[0] * Sd[0] + d[1] * Sd[1] + d[2] * Sd[2];
    *B = 2.0 * (d[0] * Sw[0] + d[1] * Sw[1] + d[2] * Sw[2]);
    *C = w[0] * Sw[0] + w[1] * Sw[1] + w[2] * Sw[2];
}

/* Euclidean distance from mu to the line c + t d (unit d). */
static double line_dist(const double mu[3], const double c[3], const double d[3]) {
    double w[3], p = 0.0, r2 = 0.0;
    for (int i = 0; i < 3; ++i) { w[i] = mu[i] - c[i]; p += w[i] * d[i]; }
    for (int i = 0; i < 3; ++i) { double e = w[i] - p * d[i]; r2 += e * e; }
    return sqrt(r2);
}

/* Euclidean distance from mu to the segment c + t d, t in [0, tmax]. */
static double segment_dist(const double mu[3], const double c[3], const double d[3], double tmax) {
    double w[3], p = 0.0, r2 = 0.0;
    for (int i = 0; i < 3; ++i) { w[i] = mu[i] - c[i]; p += w[i] * d[i]; }
    if (p < 0.0) p = 0.0;
    if (p > tmax) p = tmax;
    for (int i = 0; i < 3; ++i) { double e = w[i] - p * d[i]; r2 += e * e; }
    return sqrt(r2);
}

typedef struct {
    double t, alpha, m, A, B, C;
    int32_t g;
    int inc;  /* a hit by the FP64 decision: alpha >= 1/255 and t* > near */
    int amb;  /* that decision lies within its margin: either outcome is a correct result */
} ohit;

static int hit_cmp(const void *a, const void *b) {
    const ohit *x = (const ohit *)a, *y = (const ohit *)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return (x->g > y->g) - (x->g < y->g);  /* READING: ties broken by Gaussian index */
}

/*
 * The interval of correct results of one pixel (P11 reading: where a decision lies within its
 * margin, FP32 arithmetic may take it either way and both outcomes are correct). The sorted
 * candidate hits are composited again with every such decision taken both ways:
 *   - inclusion of a hit whose alpha lies within the margin of 1/255 or whose t* lies within the
 *     margin of the near plane,
 *   - the order of two consecutive hits whose t* lie within the order margin,
 *   - the stop, where T' lies within the margin of t_stop,
 *   - the 0.5 crossing, where T' lies within the margin of 0.5 (it is then this hit or the next).
 * Each complete sequence of decisions is a leaf; the per-channel minimum and maximum over the
 * leaves bound the correct results. More than `cap` leaves: the pixel is left unresolved.
 * The 11 channels: colour (3), depth, normal (3), opacity, exact depth, composited hit count,
 * median depth (t* of the crossing hit). An
 * exact depth whose crossing transmittance would lie at or below 0.5 (only reachable through a
 * crossing decision within its margin) is undefined: that leaf widens the exact-depth bounds to
 * (-inf, +inf).
 */
#define BR_CH 11
typedef struct {
    double T, C[3], D, N[3];
    int cnt, crossed, pend_cross;
    int kc;         /* index into the sorted hits of the crossing hit */
    double Tc;      /* transmittance in front of it */
    int first, first_forced, pend;  /* hits to process before the next in sorted order */
} bstate;

typedef struct {
    const ohit *buf;
    int nh;
    const ogauss *gs;
    const double *bg;
    double t_stop, m_tstop, m_order, m_cross;
    double lo[BR_CH], hi[BR_CH];
    int leaves, cap, over;
} bctx;

static void b_leaf(bctx *c, const bstate *s) {
    double v[BR_CH];
    for (int i = 0; i < 3; ++i) {
        v[i] = s->C[i] + s->T * (c->bg ? c->bg[i] : 0.0);
        v[4 + i] = s->N[i];
    }
    v[3] = s->D;
    v[7] = 1.0 - s->T;
    int ex_undef = 0;
    v[8] = 0.0;
    if (s->crossed) {
        const ohit *h = &c->buf[s->kc];
        const ogauss *G = &c->gs[h->g];
        if (s->Tc > 0.5) {
            double gval = (s->Tc - 0.5) / (s->Tc * G->o);
            double disc = h->B * h->B - 4.0 * h->A * (h->C + 2.0 * log(gval));
            v[8] = h->t - sqrt(disc > 0.0 ? disc : 0.0) / (2.0 * h->A);
        } else {
            ex_undef = 1;
        }
    }
    v[9] = (double)s->cnt;
    v[10] = s->crossed ? c->buf[s->kc].t : 0.0;
    for (int i = 0; i < BR_CH; ++i) {
        if (c->leaves == 0 || v[i] < c->lo[i]) c->lo[i] = v[i];
        if (c->leaves == 0 || v[i] > c->hi[i]) c->hi[i] = v[i];
    }
    if (ex_undef) {
        c->lo[8] = -INFINITY;
        c->hi[8] = INFINITY;
    }
    if (++c->leaves > c->cap) c->over = 1;
}

static int b_tie(const bctx *c, int a, int b) {
    return fabs(c->buf[b].t - c->buf[a].t) < c->m_order * c->buf[b].t;
}

static void b_run(bctx *c, int k, bstate s) {
    while (!c->over) {
        int idx, forced = 0;
        if (s.first >= 0) {
            idx = s.first;
            forced = s.first_forced;
            s.first = -1;
            s.first_forced = 0;
        } else if (s.pend >= 0) {
            idx = s.pend;
            s.pend = -1;
        } else {
            if (k >= c->nh) break;
            if (k + 1 < c->nh && b_tie(c, k, k + 1)) {
                /* the other order of a near tie: k + 1 first, then k */
                bstate s2 = s;
                s2.first = k + 1;
                s2.pend = k;
                b_run(c, k + 2, s2);
                if (c->over) return;
            }
            idx = k++;
        }
        const ohit *h = &c->buf[idx];
        if (!forced && h->amb) {
            bstate s2 = s;
            if (h->inc) {
                b_run(c, k, s2);  /* the other outcome: not a hit */
                if (c->over) return;
            } else {
                s2.first = idx;  /* the other outcome: a hit */
                s2.first_forced = 1;
                b_run(c, k, s2);
                if (c->over) return;
                continue;
            }
        }
        const double Tn = s.T * (1.0 - h->alpha);
        const int amb_stop = fabs(Tn / c->t_stop - 1.0) < c->m_tstop;
        if (Tn < c->t_stop) {
            b_leaf(c, &s);        /* stop before this hit */
            if (!amb_stop || c->over) return;
            /* the other outcome: composite it and go on */
        } else if (amb_stop) {
            b_leaf(c, &s);        /* the other outcome: stop here */
            if (c->over) return;
        }
        const ogauss *G = &c->gs[h->g];
        bstate sn = s;
        const double w = h->alpha * s.T;
        for (int i = 0; i < 3; ++i) {
            sn.C[i] += w * G->rgb[i];
            sn.N[i] += w * G->n[i];
        }
        sn.D = s.D + w * h->t;
        sn.T = Tn;
        sn.cnt = s.cnt + 1;
        if (!s.crossed) {
            const int here = s.pend_cross || (s.T > 0.5 && Tn <= 0.5);
            if (!s.pend_cross && s.T > 0.5 && fabs(Tn - 0.5) < c->m_cross * 0.5) {
                bstate alt = sn;
                if (here) {
                    alt.pend_cross = 1;  /* T' taken above 0.5: the next hit crosses */
                } else {
                    alt.crossed = 1;     /* T' taken at or below 0.5: this hit crosses */
                    alt.kc = idx;
                    alt.Tc = s.T;
                }
                b_run(c, k, alt);
                if (c->over) return;
            }
            if (here) {
                sn.crossed = 1;
                sn.pend_cross = 0;
                sn.kc = idx;
                sn.Tc = s.T;
            }
        }
        s = sn;
    }
    if (!c->over) b_leaf(c, &s);
}

/*
 * Exact-order render of selected pixels of one view.
 *   pix[n_pix]: linear pixel indices y*W+x, or NULL for all W*H pixels in row-major order.
 *   Outputs per selected pixel (any may be NULL): color[3], depth, exact_depth, median_depth,
 *   normal[3], opacity, n_contrib, flags; hits[max_hits] (composited Gaussian ids in order,
 *   -1 padded), cross_pos (index into hits of the 0.5 crossing, -1 if none), delta (distance
 *   from t* back to the exact depth at the crossing).
 *   margins[5]: relative decision margins for alpha, t_stop, near, order, crossing.
 *   slack[3] per pixel (optional): how far colour, depth and normal may move when two composited
 *   hits whose t* lie within the order margin are taken in the other order (both orders are
 *   correct results): 2 T_a alpha_a alpha_b |x_a - x_b| summed over such adjacent pairs (swapping
 *   hits a, b changes the sum by T_a alpha_a alpha_b (x_a - x_b)). An alpha within the margin of
 *   1/255 is flagged only where it could matter: at a t* before the hit that stops the pixel.
 *   cull != 0 skips Gaussians whose line distance exceeds E * s_max (cannot reach 1/255).
 *   ex_sens per pixel (optional): the change of the exact depth that FP32-sized relative errors
 *   (a few ulps) of T_k and m_k cause, plus half the order margin times t*_k (the FP32 error of
 *   t*_k, which t* - delta keeps however small it is) (0 without a crossing): its conditioning.
 *   bounds[22] per pixel (optional): the interval of correct results (b_run above), lo[11] then
 *   hi[11] over colour (3), depth, normal (3), opacity, exact depth, hit count, median depth;
 *   pixels with more
 *   than branch_cap leaves get FLAG_UNRESOLVED and bounds equal to the FP64 result.
 * Returns 0, or 1 if a pixel had more composited hits than max_hits (its list is truncated).
 */
int oracle_render(int64_t n, const float *means, const float *log_scales, const float *quats,
                  const float *logits, const float *sh, int sh_degree,
                  const float *w2c, const float *intr, int W, int H,
                  double near_plane, double t_stop, const double *bg, int cull,
                  const double *margins, const int64_t *pix, int64_t n_pix,
                  double *color, double *depth, double *exact_depth, double *median_depth,
                  double *normal, double *opacity, int32_t *n_contrib, int32_t *flags,
                  int32_t *hits, int max_hits, int32_t *cross_pos, double *delta, double *slack,
                  double *bounds, int branch_cap, double *ex_sens) {
    ocam cam;
    make_cam(w2c, intr, W, H, &cam);
    ogauss *gs = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    int64_t total = pix ? n_pix : (int64_t)W * H;
    int overflow = 0;
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g)
        prep_gauss(g, means, log_scales, quats, logits, sh, sh_degree, &cam, &gs[g]);
    double m_alpha = margins ? margins[0] : 0.0, m_tstop = margins ? margins[1] : 0.0;
    double m_near = margins ? margins[2] : 0.0, m_order = margins ? margins[3] : 0.0;
    double m_cross = margins ? margins[4] : 0.0;

#pragma omp parallel
    {
        int cap = 1024;
        ohit *buf = (ohit *)malloc(sizeof(ohit) * cap);
#pragma omp for schedule(dynamic, 16) reduction(| : overflow)
        for (int64_t ip = 0; ip < total; ++ip) {
            int64_t lin = pix ? pix[ip] : ip;
            int px = (int)(lin % W), py = (int)(lin / W);
            double d[3];
            pixel_dir(&cam, px, py, d);
            int nh = 0, fl = 0;
            double amb_t = INFINITY;  /* smallest t* of a Gaussian whose alpha is within the margin */
            for (int64_t g = 0; g < n; ++g) {
                const ogauss *G = &gs[g];
                if (!G->alive) continue;
                /* alpha >= 1/255 (1 - margin) needs m <= E^2 + 2 margin: farther lines cannot reach it */
                if (cull && line_dist(G->mu, cam.c, d) > sqrt(G->E2 + 2.0 * m_alpha) * G->smax * (1.0 + 1e-9))
                    continue;
                double A, B, C;
                ray_quadratic(G, cam.c, d, &A, &B, &C);
                double tstar = -B / (2.0 * A);            /* Eq. 9 */
                double m = C - B * B / (4.0 * A);         /* exponent of Eq. 10 */
                double alpha = fmin(ALPHA_MAX, G->o * exp(-0.5 * m));
                const int amb_alpha = fabs(alpha * 255.0 - 1.0) < m_alpha;
                const int amb_near = fabs(tstar - near_plane) < m_near * near_plane;
                if (amb_alpha && tstar > near_plane * (1.0 - m_near) && tstar < amb_t)
                    amb_t = tstar;
                if (alpha >= ALPHA_MIN && amb_near) fl |= FLAG_NEAR;
                const int inc = alpha >= ALPHA_MIN && tstar > near_plane;
                /* the enumeration of correct results also needs the hits that are ambiguous */
                const int amb = (amb_alpha && (tstar > near_plane || amb_near)) ||
                                (amb_near && (alpha >= ALPHA_MIN || amb_alpha));
                if (!inc && !(bounds && amb)) continue;
                if (nh == cap) { cap *= 2; buf = (ohit *)realloc(buf, sizeof(ohit) * cap); }
                buf[nh].t = tstar; buf[nh].alpha = alpha; buf[nh].m = m;
                buf[nh].A = A; buf[nh].B = B; buf[nh].C = C; buf[nh].g = (int32_t)g;
                buf[nh].inc = inc; buf[nh].amb = amb;
                ++nh;
            }
            qsort(buf, nh, sizeof(ohit), hit_cmp);
            /* with bounds, the list also holds the ambiguous non-hits; the FP64 result skips them */
            int nbuf = nh, ninc = 0;
            for (int k = 0; k < nbuf; ++k)
                if (buf[k].inc) ++ninc;
            ohit *hb = buf;
            ohit *inc_buf = NULL;
            if (ninc != nbuf) {
                inc_buf = (ohit *)malloc(sizeof(ohit) * (size_t)(ninc > 0 ? ninc : 1));
                int j = 0;
                for (int k = 0; k < nbuf; ++k)
                    if (buf[k].inc) inc_buf[j++] = buf[k];
                hb = inc_buf;
            }
            nh = ninc;
            double T = 1.0, Cc[3] = {0, 0, 0}, D = 0.0, Nn[3] = {0, 0, 0};
            double T_prev = 1.0, sl[3] = {0, 0, 0}, t_end = INFINITY;
            int cnt = 0, kcross = -1;
            double tcross = 0.0, dl = 0.0, sens_px = 0.0;
            for (int k = 0; k < nh; ++k) {
                const ohit *h = &hb[k];
                const ogauss *G = &gs[h->g];
                double Tn = T * (1.0 - h->alpha);
                if (fabs(Tn / t_stop - 1.0) < m_tstop) fl |= FLAG_TSTOP;
                const int near_tie = k > 0 && fabs(h->t - hb[k - 1].t) < m_order * h->t;
                if (near_tie) {
                    /* the previous hit a and this hit b may come in either order */
                    fl |= FLAG_ORDER;
                    const ohit *a = &hb[k - 1];
                    const ogauss *Ga = &gs[a->g];
                    const double f = 2.0 * T_prev * a->alpha * h->alpha;
                    double dc = 0.0, dn = 0.0;
                    for (int i = 0; i < 3; ++i) {
                        dc = fmax(dc, fabs(Ga->rgb[i] - G->rgb[i]));
                        dn = fmax(dn, fabs(Ga->n[i] - G->n[i]));
                    }
                    sl[0] += f * dc;
                    sl[1] += f * fabs(a->t - h->t);
                    sl[2] += f * dn;
                    if (Tn < t_stop) fl |= FLAG_TSTOP;          /* the swap could move the stop */
                    if (kcross >= 0 && kcross == cnt - 1) fl |= FLAG_CROSS;  /* a was the crossing */
                }
                if (Tn < t_stop) {
                    t_end = h->t;
                    break;  /* READING: stop before compositing the hit that would push T below the
                               threshold */
                }
                double w = h->alpha * T;
                for (int i = 0; i < 3; ++i) { Cc[i] += w * G->rgb[i]; Nn[i] += w * G->n[i]; }
                D += w * h->t;
                /* T' within the margin of 0.5 on a hit that does not cross: FP32 may cross here */
                if (kcross < 0 && T > 0.5 && Tn > 0.5 && fabs(Tn - 0.5) < m_cross * 0.5) fl |= FLAG_CROSS;
                if (kcross < 0 && T > 0.5 && Tn <= 0.5) {
                    /* Exact depth, Sec. 3.2 / App. A.3. READING: the defining condition
                     * T_k (1 - o_k G(t)) = 0.5 gives G(t) = (T_k - 0.5) / (T_k o_k); the root on
                     * the camera side of t* is taken. */
                    if (fabs(Tn - 0.5) < m_cross * 0.5 || fabs(T - 0.5) < m_cross * 0.5) fl |= FLAG_CROSS;
                    double gval = (T - 0.5) / (T * G->o);
                    double disc = h->B * h->B - 4.0 * h->A * (h->C + 2.0 * log(gval));
                    dl = sqrt(disc > 0.0 ? disc : 0.0) / (2.0 * h->A);
                    tcross = h->t;
                    kcross = cnt;
                    /* delta = sqrt(x/A), x = -2 ln g - m: a relative error e in T moves x by
                     * 2 e T/(T - 0.5) / 2, one in m by e m; both reach delta through
                     * 1/(2 sqrt(x A)). Flag the crossing when FP32-sized errors (e = 5e-7, a few
                     * ulps) could move the exact depth by more than half its 1e-4 relative
                     * tolerance: FP32 inputs cannot resolve it. */
                    double xq = disc / (4.0 * h->A);
                    double sens = (1e-6 * T / fabs(T - 0.5) + 1e-6 * (1.0 + fabs(h->m)) +
                                   2.4e-7 * fabs(log(gval))) / (2.0 * sqrt(fmax(xq * h->A, 1e-300)));
                    if (sens > 5e-5 * fabs(tcross - dl)) fl |= FLAG_EXACT;
                    /* the exact depth t* - delta also carries the FP32 error of t* itself, bounded
                     * by the order margin (relative to t*): it dominates where delta nearly
                     * cancels t*, i.e. where the crossing lies close to the camera */
                    sens_px = sens + 0.5 * m_order * h->t;
                    if (near_tie) fl |= FLAG_CROSS;  /* b is the crossing and may swap with a */
                }
                if (hits) {
                    if (cnt < max_hits) hits[ip * max_hits + cnt] = h->g;
                    else { overflow = 1; fl |= FLAG_OVERFLOW; }
                }
                ++cnt;
                T_prev = T;
                T = Tn;
            }
            if (amb_t < INFINITY && amb_t <= t_end) fl |= FLAG_ALPHA;  /* an ambiguous alpha before the stop */
            if (bounds) {
                double *bo = bounds + ip * 2 * BR_CH;
                /* the FP64 result, which is one of the correct results */
                const double ex0 = kcross >= 0 ? tcross - dl : 0.0;
                const double v0[BR_CH] = {Cc[0] + T * (bg ? bg[0] : 0.0), Cc[1] + T * (bg ? bg[1] : 0.0),
                                          Cc[2] + T * (bg ? bg[2] : 0.0), D, Nn[0], Nn[1], Nn[2], 1.0 - T, ex0,
                                          (double)cnt, kcross >= 0 ? tcross : 0.0};
                for (int i = 0; i < BR_CH; ++i) bo[i] = bo[BR_CH + i] = v0[i];
                if (fl & (FLAG_ALPHA | FLAG_TSTOP | FLAG_NEAR | FLAG_ORDER | FLAG_CROSS)) {
                    bctx bc;
                    memset(&bc, 0, sizeof(bc));
                    bc.buf = buf; bc.nh = nbuf; bc.gs = gs; bc.bg = bg;
                    bc.t_stop = t_stop; bc.m_tstop = m_tstop; bc.m_order = m_order; bc.m_cross = m_cross;
                    bc.cap = branch_cap;
                    bstate s0;
                    memset(&s0, 0, sizeof(s0));
                    s0.T = 1.0;
                    s0.first = s0.pend = -1;
                    b_run(&bc, 0, s0);
                    if (bc.over) {
                        fl |= FLAG_UNRESOLVED;
                    } else {
                        for (int i = 0; i < BR_CH; ++i) {
                            bo[i] = fmin(bo[i], bc.lo[i]);
                            bo[BR_CH + i] = fmax(bo[BR_CH + i], bc.hi[i]);
                        }
                    }
                }
            }
            free(inc_buf);
            if (slack) for (int i = 0; i < 3; ++i) slack[ip * 3 + i] = sl[i];
            if (hits) for (int k = cnt; k < max_hits; ++k) hits[ip * max_hits + k] = -1;
            if (color) for (int i = 0; i < 3; ++i) color[ip * 3 + i] = Cc[i] + T * (bg ? bg[i] : 0.0);
            if (depth) depth[ip] = D;
            if (normal) for (int i = 0; i < 3; ++i) normal[ip * 3 + i] = Nn[i];
            if (opacity) opacity[ip] = 1.0 - T;
            /* READING: no 0.5 crossing -> exact and median depth are 0 */
            if (exact_depth) exact_depth[ip] = kcross >= 0 ? tcross - dl : 0.0;
            if (median_depth) median_depth[ip] = kcross >= 0 ? tcross : 0.0;
            if (n_contrib) n_contrib[ip] = cnt;
            if (flags) flags[ip] = fl;
            if (cross_pos) cross_pos[ip] = kcross;
            if (delta) delta[ip] = kcross >= 0 ? dl : 0.0;
            if (ex_sens) ex_sens[ip] = sens_px;
        }
        free(buf);
    }
    free(gs);
    return overflow;
}

/*
 * Frozen-decision evaluation for finite differences: composites, for each selected pixel, exactly
 * the Gaussians listed in hits (in that order), with no hit test, no sort and no stop; the exact
 * depth at list position cross_pos uses delta_frozen (the exact-depth offset is detached in the
 * method's backward, App. A.3 "Backward Details") or, if delta_frozen is NULL, is re-solved.
 * gs: prepared Gaussians.
 */
static void frozen_core(const ogauss *gs, const ocam *cam, const double *bg, const int64_t *pix,
                        int64_t total, const int32_t *hits, int max_hits, const int32_t *cross_pos,
                        const double *delta_frozen, double *color, double *depth, double *exact_depth,
                        double *median_depth, double *normal, double *opacity) {
    int W = cam->W;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t ip = 0; ip < total; ++ip) {
        int64_t lin = pix ? pix[ip] : ip;
        int px = (int)(lin % W), py = (int)(lin / W);
        double d[3];
        pixel_dir(cam, px, py, d);
        double T = 1.0, Cc[3] = {0, 0, 0}, D = 0.0, Nn[3] = {0, 0, 0}, ex = 0.0, med = 0.0;
        for (int k = 0; k < max_hits; ++k) {
            int32_t g = hits[ip * max_hits + k];
            if (g < 0) break;
            const ogauss *G = &gs[g];
            double A, B, C;
            ray_quadratic(G, cam->c, d, &A, &B, &C);
            double tstar = -B / (2.0 * A);
            double m = C - B * B / (4.0 * A);
            double alpha = fmin(ALPHA_MAX, G->o * exp(-0.5 * m));
            double w = alpha * T;
            for (int i = 0; i < 3; ++i) { Cc[i] += w * G->rgb[i]; Nn[i] += w * G->n[i]; }
            D += w * tstar;
            if (cross_pos && k == cross_pos[ip]) {
                double dl;
                if (delta_frozen) dl = delta_frozen[ip];
                else {
                    double gval = (T - 0.5) / (T * G->o);
                    double disc = B * B - 4.0 * A * (C + 2.0 * log(gval));
                    dl = sqrt(disc > 0.0 ? disc : 0.0) / (2.0 * A);
                }
                ex = tstar - dl;
                med = tstar;
            }
            T *= (1.0 - alpha);
        }
        if (color) for (int i = 0; i < 3; ++i) color[ip * 3 + i] = Cc[i] + T * (bg ? bg[i] : 0.0);
        if (depth) depth[ip] = D;
        if (normal) for (int i = 0; i < 3; ++i) normal[ip * 3 + i] = Nn[i];
        if (opacity) opacity[ip] = 1.0 - T;
        if (exact_depth) exact_depth[ip] = ex;
        if (median_depth) median_depth[ip] = med;
    }
}

int oracle_render_frozen(int64_t n, const float *means, const float *log_scales, const float *quats,
                         const float *logits, const float *sh, int sh_degree,
                         const float *w2c, const float *intr, int W, int H, const double *bg,
                         const int64_t *pix, int64_t n_pix, const int32_t *hits, int max_hits,
                         const int32_t *cross_pos, const double *delta_frozen,
                         double *color, double *depth, double *exact_depth, double *median_depth,
                         double *normal, double *opacity) {
    ocam cam;
    make_cam(w2c, intr, W, H, &cam);
    ogauss *gs = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    for (int64_t g = 0; g < n; ++g)
        prep_gauss(g, means, log_scales, quats, logits, sh, sh_degree, &cam, &gs[g]);
    frozen_core(gs, &cam, bg, pix, pix ? n_pix : (int64_t)W * H, hits, max_hits, cross_pos, delta_frozen,
                color, depth, exact_depth, median_depth, normal, opacity);
    free(gs);
    return 0;
}

/*
 * Distortion and extent losses per pixel (Sec. 3.3 "Distortion Loss", "Extent Loss"; App. C.1,
 * C.2) over the hits a pixel composited, in the listed order (hits, as oracle_render returns them):
 *   w_i = alpha_i T_i, d_i = NDC(t*_i) = far (t*_i - near) / ((far - near) t*_i),
 *   distortion = sum_i sum_{j<i} w_i w_j (d_i - d_j)^2            (READING, see below),
 *   extent = near far / (far - near) sum_i w_i eps_i / t*_i^2,
 *   eps_i = sqrt(B^2 - 4 A (C - E^2)) / (2 A), the distance from t* at which alpha falls to 1/255.
 * near = 0.2 and far = 100 are the paper's NDC planes. READING: the loss is the pair sum over j < i,
 * the form the paper's reformulation (sum_i w_i (d_i^2 A_{i-1} + D2_{i-1} - 2 d_i D_{i-1})) and its
 * dL/dw_k equal; the symmetric double sum is twice it. NDC maps [near, far] to [0, 1], the map
 * whose derivative near far / ((far - near) t^2) the extent loss's linearisation uses.
 */
#define NDC_NEAR 0.2
#define NDC_FAR 100.0
static void loss_core(const ogauss *gs, const ocam *cam, const int64_t *pix, int64_t total, const int32_t *hits,
                      int max_hits, double *distortion, double *extent) {
    int W = cam->W;
#pragma omp parallel
    {
        double *wd = (double *)malloc(sizeof(double) * 2 * (size_t)(max_hits > 0 ? max_hits : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t ip = 0; ip < total; ++ip) {
            int64_t lin = pix ? pix[ip] : ip;
            int px = (int)(lin % W), py = (int)(lin / W);
            double d[3];
            pixel_dir(cam, px, py, d);
            double T = 1.0, ext = 0.0;
            int nk = 0;
            for (int k = 0; k < max_hits; ++k) {
                int32_t g = hits[ip * max_hits + k];
                if (g < 0) break;
                const ogauss *G = &gs[g];
                double A, B, C;
                ray_quadratic(G, cam->c, d, &A, &B, &C);
                double tstar = -B / (2.0 * A);
                double m = C - B * B / (4.0 * A);
                double alpha = fmin(ALPHA_MAX, G->o * exp(-0.5 * m));
                double w = alpha * T;
                double disc = B * B - 4.0 * A * (C - G->E2);
                double eps = sqrt(disc > 0.0 ? disc : 0.0) / (2.0 * A);
                ext += w * eps / (tstar * tstar);
                wd[2 * nk] = w;
                wd[2 * nk + 1] = NDC_FAR * (tstar - NDC_NEAR) / ((NDC_FAR - NDC_NEAR) * tstar);
                ++nk;
                T *= (1.0 - alpha);
            }
            double dist = 0.0;
            for (int i = 0; i < nk; ++i)
                for (int j = 0; j < i; ++j) {
                    double dd = wd[2 * i + 1] - wd[2 * j + 1];
                    dist += wd[2 * i] * wd[2 * j] * dd * dd;
                }
            if (distortion) distortion[ip] = dist;
            if (extent) extent[ip] = NDC_NEAR * NDC_FAR / (NDC_FAR - NDC_NEAR) * ext;
        }
        free(wd);
    }
}

int oracle_losses(int64_t n, const float *means, const float *log_scales, const float *quats, const float *logits,
                  const float *w2c, const float *intr, int W, int H, const int64_t *pix, int64_t n_pix,
                  const int32_t *hits, int max_hits, double *distortion, double *extent) {
    ocam cam;
    make_cam(w2c, intr, W, H, &cam);
    ogauss *gs = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    for (int64_t g = 0; g < n; ++g) prep_gauss(g, means, log_scales, quats, logits, NULL, 0, &cam, &gs[g]);
    loss_core(gs, &cam, pix, pix ? n_pix : (int64_t)W * H, hits, max_hits, distortion, extent);
    free(gs);
    return 0;
}

/* As oracle_render_frozen, with FP64 parameters (for finite differences below FP32 resolution). */
int oracle_render_frozen_f64(int64_t n, const double *means, const double *log_scales, const double *quats,
                             const double *logits, const double *sh, int sh_degree,
                             const float *w2c, const float *intr, int W, int H, const double *bg,
                             const int64_t *pix, int64_t n_pix, const int32_t *hits, int max_hits,
                             const int32_t *cross_pos, const double *delta_frozen,
                             double *color, double *depth, double *exact_depth, double *median_depth,
                             double *normal, double *opacity) {
    ocam cam;
    make_cam(w2c, intr, W, H, &cam);
    int K = (sh_degree + 1) * (sh_degree + 1);
    ogauss *gs = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    for (int64_t g = 0; g < n; ++g)
        prep_gauss_d(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], sh + g * K * 3, sh_degree,
                     &cam, &gs[g]);
    frozen_core(gs, &cam, bg, pix, pix ? n_pix : (int64_t)W * H, hits, max_hits, cross_pos, delta_frozen,
                color, depth, exact_depth, median_depth, normal, opacity);
    free(gs);
    return 0;
}

/*
 * Opacity field at the exact-depth point of each pixel's ray (Sec. 3.3 "Direct Opacity Field
 * Supervision"), over the hits the pixel composited (hits as oracle_render returns them): with t the
 * pixel's exact depth (Euclidean), O = 1 - prod (1 - alpha_i(min(t*_i, t))), a hit counting where
 * alpha_i(min(t*_i, t)) >= 1/255 (Eqs. 11-12 on the pixel's ray). READING: the paper evaluates
 * O_N over all Gaussians; past the render's stop the product changes by less than t_stop, and the
 * method's own second pass reuses the render's hits. -1 where t <= 0 (no 0.5 crossing).
 */
static void opa_core(const ogauss *gs, const ocam *cam, const int64_t *pix, int64_t total, const int32_t *hits,
                     int max_hits, const double *tx, double *out) {
    int W = cam->W;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t ip = 0; ip < total; ++ip) {
        int64_t lin = pix ? pix[ip] : ip;
        int px = (int)(lin % W), py = (int)(lin / W);
        if (!(tx[ip] > 0.0)) { out[ip] = -1.0; continue; }
        double d[3];
        pixel_dir(cam, px, py, d);
        double P = 1.0;
        for (int k = 0; k < max_hits; ++k) {
            int32_t g = hits[ip * max_hits + k];
            if (g < 0) break;
            const ogauss *G = &gs[g];
            double A, B, C;
            ray_quadratic(G, cam->c, d, &A, &B, &C);
            double tstar = -B / (2.0 * A);
            double te = tstar < tx[ip] ? tstar : tx[ip];
            double alpha = fmin(ALPHA_MAX, G->o * exp(-0.5 * (A * te * te + B * te + C)));
            if (alpha >= ALPHA_MIN) P *= 1.0 - alpha;
        }
        out[ip] = 1.0 - P;
    }
}

int oracle_opa(int64_t n, const float *means, const float *log_scales, const float *quats, const float *logits,
               const float *w2c, const float *intr, int W, int H, const int64_t *pix, int64_t n_pix,
               const int32_t *hits, int max_hits, const double *tx, double *out) {
    ocam cam;
    make_cam(w2c, intr, W, H, &cam);
    ogauss *gs = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    for (int64_t g = 0; g < n; ++g) prep_gauss(g, means, log_scales, quats, logits, NULL, 0, &cam, &gs[g]);
    opa_core(gs, &cam, pix, pix ? n_pix : (int64_t)W * H, hits, max_hits, tx, out);
    free(gs);
    return 0;
}

int oracle_opa_f64(int64_t n, const double *means, const double *log_scales, const double *quats,
                   const double *logits, const float *w2c, const float *intr, int W, int H, const int64_t *pix,
                   int64_t n_pix, const int32_t *hits, int max_hits, const double *tx, double *out) {
    ocam cam;
    make_cam(w2c, intr, W, H, &cam);
    ogauss *gs = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    const double zero_sh[3] = {0.0, 0.0, 0.0};
    for (int64_t g = 0; g < n; ++g)
        prep_gauss_d(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], zero_sh, 0, &cam, &gs[g]);
    opa_core(gs, &cam, pix, pix ? n_pix : (int64_t)W * H, hits, max_hits, tx, out);
    free(gs);
    return 0;
}

/* As oracle_losses, with FP64 parameters (finite differences of the loss channels). */
int oracle_losses_f64(int64_t n, const double *means, const double *log_scales, const double *quats,
                      const double *logits, const float *w2c, const float *intr, int W, int H, const int64_t *pix,
                      int64_t n_pix, const int32_t *hits, int max_hits, double *distortion, double *extent) {
    ocam cam;
    make_cam(w2c, intr, W, H, &cam);
    ogauss *gs = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    const double zero_sh[3] = {0.0, 0.0, 0.0};
    for (int64_t g = 0; g < n; ++g)
        prep_gauss_d(means + 3 * g, log_scales + 3 * g, quats + 4 * g, logits[g], zero_sh, 0, &cam, &gs[g]);
    loss_core(gs, &cam, pix, pix ? n_pix : (int64_t)W * H, hits, max_hits, distortion, extent);
    free(gs);
    return 0;
}

/*
 * Opacity field at points, min over views (Eqs. 11-12).
 *   cams: w2c[V*12], intr[V*4], wh[V*2].
 *   A view sees x iff its camera-space z exceeds the near plane and its projection lies in
 *   [0,W) x [0,H) (READING). For a seeing view, with t = |x - c| and d = (x - c)/t, every live
 *   Gaussian contributes alpha = min(0.99, o G(t_eval)), t_eval = min(t*, t), if alpha >= 1/255
 *   and t* > near; O_v = 1 - prod(1 - alpha) (order-free, App. A.2). The result is the min over
 *   seeing views, 1.0 with seen = 0 if no view sees x.
 *   per_view[P*V] (optional) receives O_v, or -1 where the view does not see the point.
 *   t_stop_query > 0 stops once the running transmittance drops below it (0 = exact).
 *   range[P*2] (optional): the interval of correct results when decisions lie within the margins:
 *   a Gaussian whose alpha is within the margin of 1/255 (or whose t* is within the margin of the
 *   near plane) may or may not be included, which moves O_v by at most its alpha; a view whose
 *   projection of x lies within the margin of the frustum may or may not see x. Then
 *   range = [min over possibly seeing views of (O_v - u_v), min over surely seeing views of
 *   (O_v + u_v)], u_v the sum of the ambiguous alphas; maybe_seen[P] (optional) counts the views
 *   whose visibility is ambiguous.
 */
int oracle_query(int64_t n, const float *means, const float *log_scales, const float *quats,
                 const float *logits, int n_views, const float *w2c, const float *intr,
                 const int32_t *wh, double near_plane, double t_stop_query, int cull,
                 const double *margins, const float *points, int64_t n_points,
                 double *opacity_out, int32_t *seen_out, double *per_view, int32_t *flags,
                 double *range, int32_t *maybe_seen) {
    ocam *cams = (ocam *)malloc(sizeof(ocam) * (size_t)(n_views > 0 ? n_views : 1));
    ogauss *gs = (ogauss *)malloc(sizeof(ogauss) * (size_t)(n > 0 ? n : 1));
    for (int v = 0; v < n_views; ++v) make_cam(w2c + v * 12, intr + v * 4, wh[v * 2], wh[v * 2 + 1], &cams[v]);
    /* geometry does not depend on the view; colour is not needed */
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g)
        prep_gauss(g, means, log_scales, quats, logits, NULL, 0, &cams[0], &gs[g]);
    double m_alpha = margins ? margins[0] : 0.0, m_near = margins ? margins[2] : 0.0;
    double m_view = margins ? margins[4] : 0.0;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t ip = 0; ip < n_points; ++ip) {
        double x[3] = {points[ip * 3], points[ip * 3 + 1], points[ip * 3 + 2]};
        double best = 1.0, lo = 1.0, hi = 1.0;
        int seen = 0, fl = 0, maybe = 0;
        for (int v = 0; v < n_views; ++v) {
            const ocam *cam = &cams[v];
            double xc[3];
            for (int i = 0; i < 3; ++i)
                xc[i] = cam->R[i][0] * x[0] + cam->R[i][1] * x[1] + cam->R[i][2] * x[2] + cam->t[i];
            int vis = 0, amb_view = 0;
            if (xc[2] > near_plane) {
                double X = cam->fx * xc[0] / xc[2] + cam->cx, Y = cam->fy * xc[1] / xc[2] + cam->cy;
                vis = X >= 0.0 && X < cam->W && Y >= 0.0 && Y < cam->H;
                double e = m_view * (1.0 + fabs(X) + fabs(Y));
                if (fabs(X) < e || fabs(X - cam->W) < e || fabs(Y) < e || fabs(Y - cam->H) < e) amb_view = 1;
            }
            if (fabs(xc[2] - near_plane) < m_near * near_plane) amb_view = 1;
            if (amb_view) { fl |= FLAG_VIEW; ++maybe; }
            if (!vis && !amb_view) { if (per_view) per_view[ip * n_views + v] = -1.0; continue; }
            double d[3], t = 0.0;
            for (int i = 0; i < 3; ++i) { d[i] = x[i] - cam->c[i]; t += d[i] * d[i]; }
            t = sqrt(t);
            for (int i = 0; i < 3; ++i) d[i] /= t;
            double P = 1.0, u = 0.0;
            for (int64_t g = 0; g < n; ++g) {
                const ogauss *G = &gs[g];
                if (!G->alive) continue;
                if (cull && segment_dist(G->mu, cam->c, d, t) > sqrt(G->E2 + 2.0 * m_alpha) * G->smax * (1.0 + 1e-9))
                    continue;
                double A, B, C;
                ray_quadratic(G, cam->c, d, &A, &B, &C);
                double tstar = -B / (2.0 * A);
                double te = tstar < t ? tstar : t;
                double alpha = fmin(ALPHA_MAX, G->o * exp(-0.5 * (A * te * te + B * te + C)));
                const int amb_a = fabs(alpha * 255.0 - 1.0) < m_alpha && tstar > near_plane * (1.0 - m_near);
                const int amb_n = alpha >= ALPHA_MIN && fabs(tstar - near_plane) < m_near * near_plane;
                if (amb_a) fl |= FLAG_ALPHA;
                if (amb_n) fl |= FLAG_NEAR;
                if (amb_a || amb_n) u += alpha;
                if (alpha >= ALPHA_MIN && tstar > near_plane) {
                    P *= (1.0 - alpha);
                    if (t_stop_query > 0.0 && P < t_stop_query) break;
                }
            }
            double Ov = 1.0 - P;
            lo = fmin(lo, fmax(Ov - u, 0.0));
            if (!amb_view) hi = fmin(hi, fmin(Ov + u, 1.0));
            if (!vis) { if (per_view) per_view[ip * n_views + v] = -1.0; continue; }
            if (per_view) per_view[ip * n_views + v] = Ov;
            if (Ov < best) best = Ov;
            seen++;
        }
        opacity_out[ip] = best;
        if (seen_out) seen_out[ip] = seen;
        if (flags) flags[ip] = fl;
        if (range) { range[ip * 2] = lo; range[ip * 2 + 1] = hi; }
        if (maybe_seen) maybe_seen[ip] = maybe;
    }
    free(cams);
    free(gs);
    return 0;
}

/*
 * Single ray/Gaussian evaluation for the pin tests: given world-space c and unit d, returns
 * out[8] = {A, B, C, t*, m (= C - B^2/4A), m via the cross-product form |o_g x d_g|^2/|d_g|^2
 * in Gaussian space (Sec. 3.1, o_g = S^-1 R^T (c - mu), d_g = S^-1 R^T d), o, E^2}.
 */
int oracle_eval_ray(const float *mean, const float *log_scale, const float *quat, float logit,
                    const double *c, const double *d, double *out) {
    ocam cam;
    memset(&cam, 0, sizeof(cam));
    for (int i = 0; i < 3; ++i) cam.c[i] = c[i];
    ogauss G;
    prep_gauss(0, mean, log_scale, quat, &logit, NULL, 0, &cam, &G);
    double A, B, C;
    ray_quadratic(&G, c, d, &A, &B, &C);
    double og[3], dg[3];
    for (int k = 0; k < 3; ++k) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 3; ++i) { a += G.Rg[i][k] * (c[i] - G.mu[i]); b += G.Rg[i][k] * d[i]; }
        og[k] = a / G.s[k]; dg[k] = b / G.s[k];
    }
    double cr[3] = {og[1] * dg[2] - og[2] * dg[1], og[2] * dg[0] - og[0] * dg[2], og[0] * dg[1] - og[1] * dg[0]};
    out[0] = A; out[1] = B; out[2] = C;
    out[3] = -B / (2.0 * A);
    out[4] = C - B * B / (4.0 * A);
    out[5] = (cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) / (dg[0] * dg[0] + dg[1] * dg[1] + dg[2] * dg[2]);
    out[6] = G.o;
    out[7] = G.E2;
    return 0;
}

/* Per-Gaussian colour and normal for one camera (for pin tests of the SH/normal readings). */
int oracle_gauss_attrs(int64_t n, const float *means, const float *log_scales, const float *quats,
                       const float *logits, const float *sh, int sh_degree, const float *w2c,
                       const float *intr, double *rgb, double *normal, double *opacity, double *E2) {
    ocam cam;
    make_cam(w2c, intr, 1, 1, &cam);
    for (int64_t g = 0; g < n; ++g) {
        ogauss G;
        prep_gauss(g, means, log_scales, quats, logits, sh, sh_degree, &cam, &G);
        for (int i = 0; i < 3; ++i) {
            if (rgb) rgb[g * 3 + i] = G.rgb[i];
            if (normal) normal[g * 3 + i] = G.n[i];
        }
        if (opacity) opacity[g] = G.o;
        if (E2) E2[g] = G.E2;
    }
    return 0;
}
