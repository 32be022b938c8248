/*
 * sof.h -- C-ABI of the GB300 (sm_103a) compositing core of Sorted Opacity Fields
 * (arXiv 2506.19139).
 *
 * The library renders 3D Gaussians by exactly depth-sorted, per-pixel, front-to-back alpha
 * compositing of their 3D-evaluated peak response along each camera ray, and evaluates the
 * opacity field at 3D points (min over views). Every entry point below is a thin host-side
 * driver of hand-written CUDA kernels; no step runs on the CPU.
 *
 * Conventions shared by all calls
 *   - Pointers documented as "device" point to GPU memory that the caller owns (for example
 *     PyTorch tensors); they must stay valid until the work queued on `stream` has finished.
 *     Pointers documented as "host" are read before the call returns.
 *   - All floating-point data is FP32, C-contiguous.
 *   - The library never allocates device memory. Scratch memory comes from a caller-provided
 *     workspace (sof_workspace_bind). If the workspace is too small the call returns
 *     SOF_ERR_WORKSPACE_TOO_SMALL and sof_workspace_required() reports the size needed.
 *   - Calls are asynchronous on `stream` except where stated. sof_render_fwd and sof_render_bwd
 *     are stream-ordered: they queue work and return, sizing their buffers from the bound
 *     workspace. Only the workspace helpers synchronise: sof_workspace_reserve (which sizes a
 *     workspace for a scene and its views), sof_workspace_stats and sof_workspace_timing; so do a
 *     forward with SOF_FLAG_CHECKED, sof_autotune, sof_graph_capture, and sof_opacity_query once
 *     per view unless SOF_QUERY_ASYNC.
 *   - Return value: 0 (SOF_OK) on success, a negative SOF_ERR_* code on failure, a positive
 *     SOF_WARN_* code when the result is valid but a warning applies. The outputs of a failed call
 *     are unspecified. sof_error_string() names every code.
 *   - Thread safety: a workspace must not be used by two calls at once; different workspaces
 *     may be used concurrently on different streams.
 *
 * Scene (Sec. 3.1 "Preliminaries"): N Gaussians with mean mu, per-axis scale s = exp(log_scale),
 * rotation R from a quaternion (w,x,y,z), normalised, with Sigma = R S S^T R^T; opacity
 * o = sigmoid(opacity_logit); colour from real spherical harmonics of degree <= 3 evaluated along
 * normalize(mu - camera centre), plus 0.5, clamped at 0.
 *
 * Camera: pinhole, world_to_cam = [R_c | t_c] row-major 3x4, OpenCV axes (x right, y down,
 * z forward). Pixel (x, y) has its centre at (x + 0.5, y + 0.5); its ray direction is
 * R_c^T ((x + 0.5 - cx)/fx, (y + 0.5 - cy)/fy, 1), normalised; ray distances are Euclidean.
 */
#ifndef SOF_H
#define SOF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------------- status codes */
#define SOF_OK 0
#define SOF_WARN_INEXACT 1                 /* reserved: a hit arrived behind one already composited
                                              (sof_stats.inexact_pixels; 0 when the path is
                                              correct, pixels whose buffer overflows are
                                              recomputed exactly instead) */
#define SOF_ERR_INVALID_ARG (-1)           /* a NULL required pointer, n < 0, bad size or option */
#define SOF_ERR_CUDA (-2)                  /* a CUDA runtime call failed (see sof_last_cuda_error) */
#define SOF_ERR_WORKSPACE_TOO_SMALL (-3)   /* bind a larger workspace and call again */
#define SOF_ERR_NOT_IMPLEMENTED (-4)
#define SOF_ERR_NO_DEVICE (-5)             /* no CUDA device of compute capability 10.3 */
#define SOF_ERR_STATE (-6)                 /* sof_render_bwd without a matching forward */

/* --------------------------------------------------------------------------------- limits */
#define SOF_MAX_VIEWS 128                  /* views per call (camera array is passed by value) */
#define SOF_MAX_SH_DEGREE 3

/* --------------------------------------------------------------------------------- inputs */
typedef struct sof_scene {
    const float *means;          /* device [n,3] */
    const float *log_scales;     /* device [n,3]: s = exp(log_scale) */
    const float *quats;          /* device [n,4] (w,x,y,z), any non-zero length */
    const float *opacity_logits; /* device [n]: o = 1/(1+exp(-logit)) */
    const float *sh;             /* device [n,(sh_degree+1)^2,3] real-SH colour coefficients */
    int64_t n;                   /* number of Gaussians, >= 0 */
    int32_t sh_degree;           /* 0..3 */
} sof_scene;

typedef struct sof_camera {
    float world_to_cam[12];      /* row-major [R_c | t_c], R_c a rotation */
    float fx, fy, cx, cy;        /* pixels */
    int32_t width, height;       /* > 0 */
} sof_camera;

/* render option flags */
#define SOF_FLAG_MEDIAN_DEPTH 1u   /* also write the median depth (t* of the 0.5 crossing) */
#define SOF_FLAG_APPROX_ORDER 4u   /* opt-in approximate per-pixel order: a pixel whose pending
                                      buffer (reorder_k hits) is full composites the buffer's
                                      nearest hit to make room instead of being redone exactly,
                                      like a fixed resort window. Only such pixels can differ
                                      from the exact result (sof_stats.inexact_pixels counts the
                                      pixels that composited a hit out of order). The backward
                                      follows the same order. */
#define SOF_FLAG_ASYNC 2u          /* accepted and ignored: every forward is stream-ordered
                                      unless SOF_FLAG_CHECKED is given. */
#define SOF_FLAG_CHECKED 8u        /* the forward reads its (Gaussian, tile) pair bound and its
                                      visible-record count back to the host (one synchronisation of
                                      `stream`) and returns SOF_ERR_WORKSPACE_TOO_SMALL, with
                                      sof_workspace_required() set, when the bound workspace cannot
                                      hold them. Without it the forward queues only stream work
                                      (capturable in a CUDA graph): the pair and visible-record
                                      capacities are those that the bound workspace holds (size it
                                      with sof_workspace_reserve), and what exceeds them is dropped
                                      and counted in sof_stats.n_dropped, summed over the forwards
                                      since sof_workspace_clear_dropped. A result with
                                      n_dropped > 0 is invalid and must be recomputed after the
                                      workspace has grown. */

typedef struct sof_render_opts {
    float near_plane;   /* a hit needs t* > near_plane (Euclidean); 0.2 in the paper (Sec. 3.3) */
    float t_stop;       /* stop before the hit that would drop transmittance below t_stop (1e-4) */
    float bg[3];        /* background colour blended with the final transmittance */
    int32_t tile;       /* screen tile edge in pixels: 0 (= 16), 8, 16 or 32. Instantiated
                           (tile, chunk, reorder_k): tile 16 with chunk 32/64/128 and reorder_k
                           8/16/32 (chunk 128: 16 only); tile 8 with chunk 64 and 16/32; tile 32
                           with chunk 64 and 8/16 (no second pass: overflowed pixels go to the
                           per-pixel fallback). */
    int32_t chunk;      /* records staged per shared-memory chunk: 0 (= 64) or 32/64/128 */
    int32_t reorder_k;  /* per-pixel pending-hit buffer: 0 (= 16) or 8/16/32 */
    uint32_t flags;     /* SOF_FLAG_* */
    int32_t replay_cap; /* hits per pixel that the forward records, in composite order, for the
                           backward to replay without re-sorting: 0 (= 256), 1..4096, or -1 (record
                           nothing: forward-only use; the backward then re-runs the merge). Pixels
                           with more hits are re-merged by the backward. Workspace cost:
                           tiles * replay_cap * 1 KiB. */
    int32_t sort_prefix; /* keys of each tile's list sorted before the composite: 0 (= 256), -1 (the
                            whole list), or n >= 1. A pixel stops once its transmittance falls
                            below t_stop, so it rarely reads past the front of its tile's list.
                            The front holds the smallest keys (at least sort_prefix of them); a
                            pixel still open where it ends is redone after the rest of its tile's
                            list is sorted. Every value gives the same images and gradients. */
} sof_render_opts;

/* Outputs of one render call over n_views views. View v owns the pixel range
 * [P_v, P_v + W_v H_v) with P_v = sum_{u<v} W_u H_u; a per-pixel scalar image of view v starts at
 * element P_v, a 3-channel planar image [3,H_v,W_v] at element 3 P_v. All device pointers. */
typedef struct sof_render_out {
    float *color;        /* [3,H,W] per view: sum_k w_k c_k + T_final bg                 (Eq. 1)  */
    float *depth;        /* [H,W]: sum_k w_k t*_k, expected ray distance, un-normalised        */
    float *exact_depth;  /* [H,W]: 0.5 level-set depth of Sec. 3.2, 0 where T never reaches 0.5 */
    float *median_depth; /* [H,W] or NULL: t* of the crossing hit (GOF depth), 0 if none       */
    float *normal;       /* [3,H,W]: sum_k w_k n_k, n_k the smallest-scale axis facing the camera */
    float *opacity;      /* [H,W]: 1 - T_final                                                  */
    int32_t *n_contrib;  /* [H,W]: number of composited hits                                    */
    /* Optional loss channels (Sec. 3.3, App. C.1-C.2), NULL = not computed (every instantiated
     * tile, chunk and reorder_k). Over the composited hits, with w_i = alpha_i T_i,
     * d_i = NDC(t*_i) = F (t*_i - N) / ((F - N) t*_i), N = 0.2, F = 100: */
    float *distortion;   /* [H,W]: sum_i sum_{j<i} w_i w_j (d_i - d_j)^2                           */
    float *extent;       /* [H,W]: N F / (F - N) sum_i w_i eps_i / t*_i^2, eps_i the distance from
                            t*_i at which alpha_i falls to 1/255                                 */
    /* Optional (NULL = not computed; needs replay_cap >= 0, i.e. recorded hits): the opacity field
     * at the exact-depth point c + t d of each pixel's ray (Sec. 3.3, the L_opa supervision),
     * 1 - prod (1 - alpha_i(min(t*_i, t))) over the hits the pixel composited with
     * alpha_i(min(t*_i, t)) >= 1/255; -1 where the pixel has no 0.5 crossing or more hits than
     * replay_cap. Its gradient takes the exact depth as given. */
    float *opacity_at_depth;
} sof_render_out;

/* Upstream gradients (device, same layouts as sof_render_out); any may be NULL (= zero). */
typedef struct sof_render_grad_in {
    const float *d_color, *d_depth, *d_exact_depth, *d_median_depth, *d_normal, *d_opacity;
    const float *d_distortion, *d_extent;  /* need the forward to have computed the channel */
    const float *d_opacity_at_depth;       /* idem */
} sof_render_grad_in;

/* Parameter gradients (device, same layouts as sof_scene); ACCUMULATED (+=) into. */
typedef struct sof_scene_grad {
    float *d_means, *d_log_scales, *d_quats, *d_opacity_logits, *d_sh;
} sof_scene_grad;

typedef struct sof_query_opts {
    float near_plane;    /* view sees x iff z_cam(x) > near_plane; Gaussians need t* > near_plane */
    float t_stop_query;  /* 0 = exact; > 0 stops a view once its transmittance < t_stop_query,
                            changing the result by at most t_stop_query                       */
    int32_t tile;        /* screen tile edge in pixels: 0 (= 16), 8, 16 or 32 */
    uint32_t flags;      /* SOF_QUERY_* */
} sof_query_opts;

/* query option flags */
#define SOF_QUERY_LEVEL_SET 1u /* level-set test (Sec. 3.4 "Early Stopping", the binary search):
                                  only whether O(x) > 0.5 is exact. A view stops as soon as its
                                  O_v(x) exceeds 0.5, and a point is skipped by every later view
                                  once one view gave O_v(x) <= 0.5 (O is a min over views).
                                  opacity_out[i] > 0.5 iff O(x_i) > 0.5; the values themselves
                                  are partial. */
#define SOF_QUERY_ASYNC 2u     /* no host round trip per view (capturable in a CUDA graph): the
                                  Gaussian pairs of a view are bounded by the workspace's capacity;
                                  pairs beyond it are dropped and counted in sof_stats.n_dropped
                                  (the result is then invalid). Size the workspace with a
                                  synchronous query of the same scene and views first. */

#define SOF_QUERY_PREPARED 4u   /* use the views that sof_query_prepare left resident in the workspace
                                  (same scene size, cameras, tile and near plane, else
                                  SOF_ERR_STATE): only the points' work runs, with no host round
                                  trip (capturable in a CUDA graph) */

typedef struct sof_stats {
    int64_t n_pairs;          /* (Gaussian, tile) pairs sorted in the last call           */
    int64_t n_visible;        /* (Gaussian, view) records that were not culled            */
    int64_t inexact_pixels;   /* pixels whose exact order was broken (SOF_WARN_INEXACT)   */
    int64_t nonfinite;        /* Gaussians culled because a parameter was NaN or infinite */
    int64_t n_point_views;    /* (point, view) pairs integrated in the last query         */
    int64_t n_tests;          /* (pixel, record) closed-form tests in the last forward    */
    int64_t n_hits;           /* tests with alpha >= 1/255 and t* > near                  */
    int64_t n_composited;     /* hits blended before the transmittance stop               */
    int64_t n_forced;         /* pixels recomputed by the exact overflow fallback         */
    int64_t n_below_key;      /* hits below their own record's sort key (0 when correct)  */
    int64_t n_unsorted;       /* tile streams whose keys decrease (0 when correct)        */
    int64_t n_replayed;       /* hits the last backward replayed from the recorded order  */
    int64_t n_dropped;        /* pairs or visible records beyond the capacities, summed over the
                                 forwards since sof_workspace_clear_dropped (SOF_FLAG_ASYNC only;
                                 their results are invalid unless 0); after a query, its own
                                 (SOF_QUERY_ASYNC)                                           */
    int64_t n_open;           /* pixels redone because they outlived their tile's sorted front */
    int64_t n_read;           /* tile-list entries the forward's first composite pass read     */
} sof_stats;

typedef struct sof_workspace sof_workspace;  /* opaque host handle */

/* ------------------------------------------------------------------------------ workspace */
/* Create / destroy a host handle. It owns no device memory. */
int sof_workspace_create(sof_workspace **ws);
int sof_workspace_destroy(sof_workspace *ws);

/* Bind `bytes` of caller-owned device memory (256-byte aligned) as scratch for later calls.
 * Rebinding drops the state a forward left for its backward. */
int sof_workspace_bind(sof_workspace *ws, void *device_ptr, size_t bytes);

/* Bytes a render over these views needs for `pair_capacity` (Gaussian, tile) pairs. */
int sof_render_workspace_size(const sof_scene *scene, const sof_camera *cams, int n_views,
                              const sof_render_opts *opts, int64_t pair_capacity, size_t *bytes);

/* Bytes a query needs for `pair_capacity` Gaussian pairs and `point_capacity` (point, view)
 * entries per view. */
int sof_query_workspace_size(const sof_scene *scene, const sof_camera *cams, int n_views,
                             int64_t n_points, const sof_query_opts *opts, int64_t pair_capacity,
                             size_t *bytes);

/* Sizes a workspace for renders of this scene and these views (Sec. 3.1: the per-(Gaussian, view)
 * records and the (Gaussian, tile) pair bound of the binning). Runs the preprocessing and the pair
 * bound on `stream`, waits for them, and returns in *bytes the workspace size that a stream-ordered
 * sof_render_fwd (and its sof_render_bwd) of the same scene, views and options needs, with 1/8
 * slack on the pairs. The visible-record count it saw raises the workspace's visible-record
 * capacity (it only grows, so that the several calls of a batched step can share one workspace).
 * The bound workspace must hold the records: on SOF_ERR_WORKSPACE_TOO_SMALL bind
 * sof_workspace_required() bytes and call again. Leaves no state for sof_render_bwd.
 * Errors as sof_render_fwd. */
int sof_workspace_reserve(sof_workspace *ws, const sof_scene *scene, const sof_camera *cams, int n_views,
                          const sof_render_opts *opts, void *stream, size_t *bytes);

/* After SOF_ERR_WORKSPACE_TOO_SMALL: the byte count the failed call needed. */
int sof_workspace_required(const sof_workspace *ws, size_t *bytes);

/* Counters of the last call on this workspace (synchronises the workspace's last stream). */
int sof_workspace_stats(const sof_workspace *ws, sof_stats *stats);

/* Zero the dropped-capacity counter reported by sof_workspace_stats (queued on stream; can be
 * captured in a CUDA graph together with the calls it covers). */
int sof_workspace_clear_dropped(sof_workspace *ws, void *stream);

/* Per-phase device timing. While enabled, every call on the workspace records a CUDA event pair
 * on its stream around each phase below; sof_workspace_timing() waits for the recorded events,
 * returns per phase the summed milliseconds and the number of timed launches since timing was
 * enabled (or last read), and clears them. Phases a call does not run stay 0. Enabling, disabling
 * and reading are host calls on this workspace only; errors: SOF_ERR_INVALID_ARG (null), SOF_ERR_CUDA. */
enum {
    SOF_PHASE_PREPROCESS = 0,   /* per (Gaussian, view) records                        */
    SOF_PHASE_BIN_COUNT,        /* pair bound per record (render) / pairs per record (query) */
    SOF_PHASE_SCAN,             /* exclusive scan of the per-record counts              */
    SOF_PHASE_BIN_EMIT,         /* (tile, depth key, Gaussian) pairs after the tile test */
    SOF_PHASE_SORT,             /* pairs into per-tile ranges, sorted by depth in each tile */
    SOF_PHASE_COMPOSITE,        /* exact-order composite, main kernel (forward)         */
    SOF_PHASE_FALLBACK,         /* exact fallback of overflowed pixels (forward)        */
    SOF_PHASE_REPLAY_BWD,       /* backward of pixels replaying their recorded order    */
    SOF_PHASE_COMPOSITE_BWD,    /* backward re-merge: main kernel + fallback            */
    SOF_PHASE_GRAD_REDUCE,      /* zeroing and summing the gradient copies              */
    SOF_PHASE_PREPROCESS_BWD,   /* chain rule from record gradients to the parameters   */
    SOF_PHASE_QUERY_POINTS,     /* query: point projection, keys, sort, block tables    */
    SOF_PHASE_QUERY_INTEGRATE,  /* query: per-point front-to-back opacity               */
    SOF_N_PHASES
};
int sof_workspace_set_timing(sof_workspace *ws, int enable);
int sof_workspace_timing(sof_workspace *ws, double ms[SOF_N_PHASES], int64_t launches[SOF_N_PHASES]);

/* ----------------------------------------------------------------------------- rendering */
/*
 * Forward render of n_views views (Sec. 3.1 Eqs. 1-10, Sec. 3.2 "Exact Depth").
 * Per pixel, every Gaussian whose 3D-evaluated peak response along the pixel ray gives
 * alpha = min(0.99, o exp(-m/2)) >= 1/255 and t* > near_plane is a hit; hits are composited in
 * exact ascending (t*, Gaussian index) order, front to back, stopping before the hit that would
 * drop the transmittance below t_stop. m is the minimum squared Mahalanobis distance along the
 * ray and t* the Euclidean distance of that minimum (Eqs. 9-10). exact_depth solves
 * T_k (1 - o_k G(t)) = 0.5 on the first hit k whose transmittance crosses 0.5, on the camera
 * side of t*_k (App. A.3).
 * cams: host array [n_views], 1 <= n_views <= SOF_MAX_VIEWS.
 * The workspace keeps the per-view records and sorted lists for a following sof_render_bwd.
 * Returns SOF_OK, SOF_WARN_INEXACT, or an error.
 */
int sof_render_fwd(const sof_scene *scene, const sof_camera *cams, int n_views,
                   const sof_render_opts *opts, const sof_render_out *out, sof_workspace *ws,
                   void *stream /* cudaStream_t */);

/*
 * Backward of the last sof_render_fwd on this workspace (same scene, cameras and options; `fwd`
 * must hold that call's outputs: other cameras or other output pointers return SOF_ERR_STATE). Replays the forward's per-pixel decisions front to back and
 * accumulates (+=) gradients of sum(grad_in * outputs) with respect to means, log-scales,
 * quaternions, opacity logits and SH coefficients. The exact-depth offset from t*_k to the 0.5
 * crossing is detached, as in the paper's implementation (App. A.3 "Backward Details"): the
 * gradient of exact_depth flows through t*_k only. Decisions (hit set, order, stop, crossing)
 * are piecewise constant and carry no gradient.
 */
int sof_render_bwd(const sof_scene *scene, const sof_camera *cams, int n_views,
                   const sof_render_opts *opts, const sof_render_out *fwd,
                   const sof_render_grad_in *grad_in, const sof_scene_grad *grad,
                   sof_workspace *ws, void *stream);

/* ----------------------------------------------------------------------- opacity field */
/*
 * Opacity field at points (Eqs. 11-12, App. A.2). A view sees x iff z_cam(x) > near_plane and
 * the projection of x lies in [0,W) x [0,H). For a seeing view, with t = |x - c| and d the unit
 * direction from the camera centre c to x, every Gaussian contributes
 * alpha = min(0.99, o G(t_eval)), t_eval = min(t*, t), if alpha >= 1/255 and t* > near_plane;
 * O_v(x) = 1 - prod (1 - alpha), which does not depend on order (App. A.2).
 * opacity_out[i] = min over seeing views of O_v(x_i), 1.0 if no view sees x_i.
 * seen_count[i] (optional) = number of seeing views.
 * points: device [n_points,3]; opacity_out: device [n_points]; seen_count: device [n_points] or
 * NULL. cams: host array [n_views].
 */
int sof_opacity_query(const sof_scene *scene, const sof_camera *cams, int n_views,
                      const float *points, int64_t n_points, const sof_query_opts *opts,
                      float *opacity_out, int32_t *seen_count, sof_workspace *ws, void *stream);

/*
 * Prepares queries of the opacity field over a fixed scene and set of views (Sec. 3.4 "Ray/Tile
 * Scheduling": the Gaussians of every view are bucketed by screen tile and sorted by z_min once).
 * Builds every view's query records and per-tile z_min-sorted Gaussian lists and keeps them
 * resident at the front of the workspace, so that later calls with SOF_QUERY_PREPARED (the
 * queries of one pass, the steps of a level-set bisection) do only the points' work. The lists
 * hold every tile of each view. Synchronises `stream` once per view (a counting pass sizes the
 * resident lists) and returns SOF_ERR_WORKSPACE_TOO_SMALL with sof_workspace_required() set when
 * the bound workspace cannot hold them together with the larger of the building scratch and the
 * points' scratch of a prepared query of max_points points, or of a prepared bisection of as many
 * edges (about 48 bytes per point plus per-tile tables). The resident state lasts until the
 * workspace is rebound or another call than a prepared query uses it. The scene's values are read
 * now: a prepared query sees the Gaussians as they were at preparation.
 */
int sof_query_prepare(const sof_scene *scene, const sof_camera *cams, int n_views, int64_t max_points,
                      const sof_query_opts *opts, sof_workspace *ws, void *stream);

/*
 * Binary search for the 0.5 level set of O along edges (Sec. 3.4: marching tetrahedra refine the
 * crossing with 8 bisection steps). Edge e runs from inside[e] (O > 0.5) to outside[e]
 * (O <= 0.5); each step queries the midpoint m in SOF_QUERY_LEVEL_SET mode (all edges in one
 * query) and moves inside[e] to m if O(m) > 0.5, else outside[e]. The endpoints are updated in
 * place; after `iterations` steps the crossing lies in [inside[e], outside[e]] (whose midpoint
 * is the usual answer), which is 2^-iterations of the original edge long.
 * inside, outside: device [n_edges,3], read and written. opts->flags must have
 * SOF_QUERY_LEVEL_SET. The workspace must hold a query of n_edges points plus 16 bytes per edge
 * (sof_level_set_workspace_size).
 */
int sof_level_set_bisect(const sof_scene *scene, const sof_camera *cams, int n_views, float *inside,
                         float *outside, int64_t n_edges, int iterations, const sof_query_opts *opts,
                         sof_workspace *ws, void *stream);

/* ------------------------------------------------------ batched step in a CUDA graph, autotuner */
/*
 * The batched training step (many views per step; the paper renders one view per iteration, so
 * this has no counterpart there beyond Sec. 3.1's per-view render and Sec. 3.3's backward): the
 * parameter gradients are zeroed (if zero_grads), the dropped-capacity counter is cleared, then
 * the views are rendered in groups of views_per_call (0 = all in one call), each group a
 * stream-ordered sof_render_fwd followed by its sof_render_bwd on the one workspace, the
 * gradients accumulating over the groups. sof_graph_capture captures that step into a CUDA graph;
 * sof_graph_launch replays it on any stream, reading the current contents of the scene, upstream
 * gradient buffers and writing the outputs and gradients (all device pointers fixed at capture).
 *   - out / grad_in: packed over all n_views views as in sof_render_out (view v at pixel P_v); the
 *     groups use their slices. grad: accumulated (+=), zeroed first if zero_grads.
 *   - Capture sizes the workspace first (sof_workspace_reserve per group, synchronising): if the
 *     bound workspace is too small it returns SOF_ERR_WORKSPACE_TOO_SMALL with
 *     sof_workspace_required() set; bind that and call again. It then runs the step once eagerly
 *     (outputs and gradients are written) and captures it on `stream`, which must not be the legacy
 *     default stream (NULL): SOF_ERR_INVALID_ARG.
 *   - The capacities stay those of capture time: after a launch, sof_workspace_stats().n_dropped
 *     > 0 means the step's results are invalid (the scene changed enough to need more pairs).
 *   - The graph uses the workspace: one launch at a time per workspace, and no other call on the
 *     workspace between a launch and the reading of its results.
 *   - Phase timing is off inside the graph.
 */
typedef struct sof_graph sof_graph;  /* opaque host handle */
int sof_graph_capture(const sof_scene *scene, const sof_camera *cams, int n_views, int views_per_call,
                      const sof_render_opts *opts, const sof_render_out *out, const sof_render_grad_in *grad_in,
                      const sof_scene_grad *grad, int zero_grads, sof_workspace *ws, void *stream,
                      sof_graph **graph);
int sof_graph_launch(sof_graph *graph, void *stream);
int sof_graph_destroy(sof_graph *graph);

/*
 * Autotuner of the composite's launch parameters (no counterpart in the paper). Every instantiated
 * (tile, chunk, reorder_k) triple (SOF_AUTOTUNE_CANDIDATES of them, in the order of
 * sof_autotune_candidate) renders the same exact images; the fastest depends on the scene's depth
 * complexity, the Gaussians' screen sizes and the views. Times `reps` batched steps (as in
 * sof_graph_capture, eager, after one warm-up step) of every triple on the caller's own workload with
 * CUDA events on `stream` and writes the fastest into *best (base with tile, chunk, reorder_k
 * replaced). ms (optional, [SOF_AUTOTUNE_CANDIDATES]) receives each triple's ms per step, -1 where
 * the library refuses the triple for this workload (SOF_ERR_INVALID_ARG, e.g. more candidate pairs
 * than one call indexes). out, grad_in and grad are scratch during tuning: their contents
 * afterwards are unspecified.
 *   - cache_path (optional): a text file of "signature tile chunk reorder_k ms" lines; a workload
 *     whose signature (Gaussian count, SH degree, view sizes, views per call, base options) is
 *     found returns the cached triple without timing (ms then holds -1 except at the chosen
 *     triple), else the result is appended.
 *   - The workspace must hold every triple's step: SOF_ERR_WORKSPACE_TOO_SMALL with
 *     sof_workspace_required() set otherwise (checked before anything is timed).
 *   - Synchronises `stream`.
 */
#define SOF_AUTOTUNE_CANDIDATES 11
int sof_autotune_candidate(int index, int *tile, int *chunk, int *reorder_k);
int sof_autotune(const sof_scene *scene, const sof_camera *cams, int n_views, int views_per_call,
                 const sof_render_opts *base, const sof_render_out *out, const sof_render_grad_in *grad_in,
                 const sof_scene_grad *grad, int reps, const char *cache_path, sof_workspace *ws, void *stream,
                 sof_render_opts *best, float *ms);

/* -------------------------------------------------- forward render without any allocation */
/*
 * (No counterpart in the paper: this is a deployment convenience of this library.)
 * For callers that cannot allocate device memory -- code running where cudaMalloc/cudaFree are
 * unavailable or forbidden, or where every byte of device memory was reserved up front -- this
 * entry point renders like sof_render_fwd but takes its scratch from a fixed array compiled into
 * the library (SOF_NOALLOC_SCRATCH_BYTES per device), so the call itself allocates nothing. The
 * array occupies that much memory on every GPU that loads the library until the process exits.
 *   - The caller still passes inputs and outputs (all device pointers, as for sof_render_fwd).
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current; make that first call before any stream capture.
 *   - Every call is checked (as with SOF_FLAG_CHECKED, whatever opts->flags say; it therefore
 *     synchronises `stream` once) and sized on its own, so whether a scene fits does not depend on
 *     earlier calls. Scenes whose records, (Gaussian, tile) pairs or pixels do not fit the array
 *     are rejected with SOF_ERR_WORKSPACE_TOO_SMALL, never rendered with pairs dropped;
 *     *required_bytes (if not NULL) receives the scratch size the call would have needed. Use
 *     sof_render_fwd with a caller-bound workspace for those.
 *   - It records no hits for a backward (opts->replay_cap is taken as -1), so the
 *     opacity_at_depth output is refused (SOF_ERR_INVALID_ARG).
 *   - sof_noalloc_last_error() returns the message of the calling thread's last failed call.
 *   - All calls on a device share the array and it keeps the last call's contents; every call
 *     clears what must start at zero. Calls that overlap on the GPU (different streams, or a call
 *     issued before the previous one's work finished on another stream) race on it: serialise
 *     them. The array holds no state for sof_render_bwd.
 */
#define SOF_NOALLOC_SCRATCH_BYTES (24u << 20)
int sof_render_fwd_noalloc(const sof_scene *scene, const sof_camera *cams, int n_views,
                           const sof_render_opts *opts, const sof_render_out *out,
                           size_t *required_bytes, void *stream);
const char *sof_noalloc_last_error(void);

/* --------------------------------------------------------------------------------- misc */
const char *sof_error_string(int code);
/* Number of CUDA kernels this library has launched in this process (diagnostics). */
int64_t sof_kernel_launches(void);
const char *sof_last_cuda_error(const sof_workspace *ws);
/* Roofline denominators of the per-pixel and per-point kernels, measured on the current device
 * (no counterpart in the paper): the FP32 FMA issue rate and the MUFU (ex2) rate in T operations
 * per second, each the best of three timed launches of independent dependency chains on every SM
 * (an FFMA counts as one operation). Takes about 50 ms; synchronises `stream`. */
int sof_measure_issue_peaks(double *fp32_tops, double *mufu_tops, void *stream);
int sof_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SOF_H */
