// Internal declarations of the sm_103a compositing core (not part of the public C-ABI).
//
// Data layout in HBM (per call, inside the caller-bound workspace):
//   records      [V*N][6] float4   per (view, Gaussian) render record, 96 B      (k_preprocess)
//   qrecords     [V*N][6] float4   per (view, Gaussian) query record, 96 B       (query path)
//   aux          [V*N]    float4   {t_lo_global, rho2, z_min, alive}             (k_preprocess)
//   rects        [V*N]    int4     tile rectangle [tx0,ty0,tx1,ty1) in view tiles (k_preprocess)
//   counts/offs  [V*N]    int32    (Gaussian, tile) pairs per record, exclusive scan
//   keys/vals    2 x [P]  u64/u32  (view-tile << 32 | depth-bits, record index), ping-pong sort
//   ranges       [tiles]  int2     [start, end) of each tile's run in the sorted pairs
//   rgrad        [V*N][6] float4   per-record gradients accumulated by the backward composite
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sof.h"

namespace sof {

constexpr float kAlphaMin = 1.0f / 255.0f;  // Eq. 3 cut-off
constexpr float kAlphaMax = 0.99f;          // alpha clamp
constexpr int kRecF4 = 8;                   // float4 per record (layout in record.cuh)
constexpr int kGradF4 = 6;                  // float4 per record gradient
constexpr int kGradCopies = 16;             // backward accumulates into this many copies per record

// The record layout and its per-pixel evaluation are in record.cuh.

// Per-view camera, prepared on the host in FP64 from the FP32 inputs.
struct DevCam {
    double R[9];      // world -> camera rotation (FP32 inputs, exact in FP64)
    double t[3];
    double rfx, rfy;  // 1 / fx, 1 / fy (FP64 divisions are slow on GB300: kernels multiply)
    float Rf[9];
    float tf[3];      // t (FP32 inputs)
    float cf[3];      // camera centre -R^T t, rounded to FP32
    float fx, fy, cx, cy;
    float zclip;      // no in-image pixel ray reaches Euclidean near_plane below this camera z
    int W, H;
    int tiles_x, tiles_y;
    int tile_base;    // first global tile index of this view
    long long pix_base;  // first pixel of this view in the packed output images
};

struct CamSet {
    int n_views;
    int tile;
    int total_tiles;
    int pad;
    DevCam cam[SOF_MAX_VIEWS];
};

// The camera set travels to the device as a kernel parameter (under 32 KB for SOF_MAX_VIEWS views),
// not as a copy from host memory, so that a call can be captured in a CUDA graph.
static_assert(sizeof(CamSet) <= 32000, "CamSet must fit in a kernel parameter");
cudaError_t launch_set_cams(const CamSet &cams, CamSet *dst, cudaStream_t s);
cudaError_t launch_add_u64(const unsigned long long *src, unsigned long long *dst, cudaStream_t s);
cudaError_t launch_sum64(const int *in, long long n, unsigned long long *acc, cudaStream_t s);
cudaError_t launch_guard_items(const unsigned long long *area_total, int *n_items, unsigned long long *dropped,
                               cudaStream_t s);

// Device-side counters written by the kernels (one per workspace). The frequent ones are spread
// over kCntShards copies (by CTA and warp), so that the atomics of many CTAs do not queue on one
// address; the host sums the copies.
constexpr int kCntShards = 64;
enum CountField {
    kCntTests,       // (pixel, record) closed-form tests in the composite (query: point tests)
    kCntHits,        // tests that passed alpha >= 1/255 and t* > near (query: included)
    kCntComposited,  // hits blended before the transmittance stop
    kCntRead,        // list entries the forward's first composite pass staged
    kCntReplayed,    // hits replayed by the backward from the recorded order
    kCntVisible,     // records that were not culled
    kCntPointViews,  // (point, view) pairs integrated by the query
    kCntFields = 8
};
struct DevStatus {
    unsigned long long n_pairs;
    unsigned long long inexact_pixels;
    unsigned long long nonfinite;
    unsigned long long overflow;
    unsigned long long n_forced;      // pixels recomputed by the exact fallback (buffer overflow)
    unsigned long long n_below_key;   // hits whose t*' is below their own record's key (must be 0)
    unsigned long long n_unsorted;    // tile streams whose keys decrease (must be 0)
    unsigned long long n_dropped;     // pairs or visible records beyond the capacities
    unsigned long long area_total;    // 64-bit sum of the records' tile counts (pair bound)
    unsigned long long n_open;        // pixels still open at the end of their tile's sorted front
    unsigned long long cnt[kCntShards][kCntFields];
};

__device__ __forceinline__ void add_count(DevStatus *s, int field, unsigned long long v) {
    atomicAdd(&s->cnt[(blockIdx.x * 8u + (threadIdx.x >> 5)) & (kCntShards - 1)][field], v);
}

// 1 / z in FP64 without an FP64 division (FP64 runs at a small fraction of the FP32 rate on
// GB300): a float reciprocal (relative error about 2^-23 with the rounding of z) refined by one
// Newton-Raphson step r (2 - z r), which squares the relative error to about 2^-46. Outside the
// float range the division is taken as it is.
__device__ __forceinline__ double recip_fp64(double z) {
    const float zf = (float)z;
    if (!(fabsf(zf) > 1e-30f && fabsf(zf) < 1e30f)) return 1.0 / z;
    const double r = (double)__frcp_rn(zf);
    return r * fma(-z, r, 2.0);
}

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, cached per
// device): grids of the resident and grid-stride kernels are sized in multiples of it.
int device_sm_count();

// Accessors of the opaque workspace for the host-side drivers outside api.cu.
bool workspace_timing(const sof_workspace *ws);
size_t workspace_bytes(const sof_workspace *ws);  // bound bytes (0 if unbound)
void workspace_set_required(sof_workspace *ws, size_t bytes);
void workspace_note(sof_workspace *ws, const char *msg);

// Process-wide count of kernels this library launched (diagnostics; sof_kernel_launches()).
void note_launches(long long k);

struct SceneDev {
    const float *means, *log_scales, *quats, *logits, *sh;
    long long n;
    int sh_degree;
};

// ---------------------------------------------------------------- launchers (one per .cu)
// preprocess.cu
cudaError_t launch_preprocess(const SceneDev &sc, const CamSet *cams_dev, const CamSet &cams_host,
                              float near_plane, bool query_records, float4 *records, float4 *aux,
                              int4 *rects, DevStatus *status, cudaStream_t s);
// count and emit must see the same query_keys so that they test the same tiles; emit never writes
// more than counts[rec] pairs for a record.
// scan.cu
size_t scan_temp_bytes(long long n);
cudaError_t launch_exclusive_scan(const int *in, int *out, long long n, void *temp,
                                  int *total_dev, cudaStream_t s);
// The same into 64-bit sums (the binning's item offsets of a call over many views).
cudaError_t launch_exclusive_scan64(const int *in, long long *out, long long n, void *temp, long long *total_dev,
                                    cudaStream_t s);
cudaError_t launch_rect_area(const float4 *aux, const int4 *rects, long long n_rec, int *area, int *flag,
                             cudaStream_t s);
cudaError_t launch_compact_visible(const int *area, const int *flag, const int *pos, long long n_rec, int *vis_list,
                                   int *vis_area, long long vis_cap, unsigned long long *dropped, cudaStream_t s);
// Item offsets (vis_off) and the item total are 64-bit; *cursor counts the appended pairs (64-bit;
// positions at or beyond cap are dropped and counted). ptile == nullptr: count the passing pairs
// only (block_first may be nullptr: a binary search per CTA). With prank, each appended pair's rank
// among its tile's pairs (the tile count before it) is stored beside it.
cudaError_t launch_bin_append(const CamSet *cams_dev, long long n_per_view, const float4 *records, const float4 *aux,
                              const int4 *rects, const int *vis_list, const long long *vis_off, const int *n_vis_dev,
                              const long long *n_items_dev, long long max_items, bool query_keys, float near_plane,
                              long long cap, unsigned long long *cursor, unsigned *ptile, unsigned *pkey,
                              unsigned *prec, int *tile_counts, unsigned long long *dropped, cudaStream_t s,
                              const int *block_first = nullptr, const int *tile_need = nullptr,
                              unsigned *prank = nullptr);
// block_first[b] (b < items / 256 + 1): the compacted record holding the first item of binning CTA
// b, so that k_bin_append needs no binary search over the item offsets.
cudaError_t launch_block_first(const long long *vis_off, const int *n_vis_dev, const long long *n_items_dev,
                               long long max_vis, long long max_items, int *block_first, cudaStream_t s);
// tilesort.cu
constexpr int kTileOpen = 2;

// Render lists: only the front of each tile's list is sorted up front (k_tile_select).
struct FrontSort {
    unsigned long long *out;  // [pairs] the tiles' lists: sorted front, then the rest
    int prefix;               // words per tile the front holds at least (<= 0: whole lists)
    int *prefix_end;          // [tiles] end of the sorted front
    float *prefix_key;        // [tiles] lower bound of the keys after the front (+inf: none)
    int *tile_flag;           // [tiles] zeroed here; set by the composite's first pass
};
// Buckets the unsorted (tile, key, record) lists into `pairs` by tile. Without `front` each
// tile's range is then sorted in place: up to 8192 words by a radix sort in shared memory, longer
// ones by the radix sort through `scratch` (as many words as `pairs`; it may be the unsorted
// lists' own memory, which the bucketing has finished reading) or, without it, by the bitonic
// network. blocks_only is for lists whose order only groups similar keys: the radix sorts then
// order by the key's top 16 bits alone, and the bitonic network sorts 8192-word blocks without
// merging them. With `front`, the front of each range is selected and sorted into front->out.
// With prank (each pair's rank in its tile, from the append), a pair goes to its tile's offset plus
// its rank with no atomic; without it, through an atomic cursor per tile.
cudaError_t launch_tile_buckets(const unsigned *ptile, const unsigned *pkey, const unsigned *prec,
                                const unsigned long long *n_dev, long long cap, const int *tile_counts,
                                const int *tile_offsets, int n_tiles, int2 *ranges, int *cursor,
                                unsigned long long *pairs, unsigned long long *pair_total, cudaStream_t s,
                                const FrontSort *front = nullptr, bool blocks_only = false,
                                unsigned long long *scratch = nullptr, const unsigned *prank = nullptr);
// Sorts the rest of the lists ([prefix_end[t], range.y)) of the tiles list[0, *count).
cudaError_t launch_tail_sort(const int2 *ranges, const int *prefix_end, const int *list, const int *count,
                             unsigned long long *pairs, cudaStream_t s);
// composite.cu
struct CompositeParams {
    const CamSet *cams;
    const float4 *records;
    const unsigned long long *pairs;  // per tile, ascending: depth key bits << 32 | record index
    const int2 *ranges;               // [tiles] range of each tile's pairs
    // first pass only: [tiles] end of the sorted front and the lower bound of the keys after it
    // (nullptr: the whole range is sorted)
    const int *prefix_end;
    const float *prefix_key;
    // [tiles] kTileOpen: a pixel of the tile outlived the front in the first pass, so the second
    // pass and the fallback read the whole (by then sorted) list
    int *tile_flag;
    // tiles whose rest of the list must be sorted before the next pass: the first pass appends the
    // tiles it flags, the second pass the tiles of its fallback pixels that are not flagged
    int *open_tiles[2], *open_count[2];
    // tiles with pixels left to the second pass: the first forward pass appends them, and the
    // second pass (forward and backward) runs over this list instead of every tile (nullptr: every
    // tile)
    int *redo_tiles, *redo_count;
    float near_plane, t_stop;
    float bg[3];
    float *color, *depth, *exact_depth, *median_depth, *normal, *opacity;
    int *n_contrib;
    // backward only
    const float *d_color, *d_depth, *d_exact, *d_median, *d_normal, *d_opacity;
    float4 *rgrad;      // [visible records][kGradCopies][6] gradient copies, summed afterwards
    const int *vis_pos;  // [records] compacted index of a record with tiles (rank among them)
    int vis_cap;         // visible records the gradient copies hold
    DevStatus *status;
    // pixels whose pending buffer overflowed: recomputed exactly by the fallback kernel
    unsigned char *ovf_mask;  // [pixels], written by the forward, read by the backward
    unsigned *ovf_list;       // [pixels] (global tile << 8 | thread)
    int *ovf_count;           // reset by the forward only
    int pass;                 // 0: every pixel; 1: the pixels the first pass gave up (larger buffer)
    bool approx;              // SOF_FLAG_APPROX_ORDER: a full buffer composites its nearest hit
    // distortion and extent loss channels (Sec. 3.3): outputs, upstream gradients, and the
    // forward's per-pixel sums for the backward; loss_sums == nullptr: off
    float *distortion, *extent;
    const float *d_distortion, *d_extent;
    float4 *loss_sums;  // [pixels] (sum w u, sum w u^2, sum w e, dref), u = d - dref
    // opacity field at the exact depth (k_opacity_at_depth): the output / the forward's output in
    // the backward, and its upstream gradient
    float *opa;
    const float *d_opa;
    unsigned *ovf_list2;      // [pixels] pixels the second pass gave up: the per-pixel fallback's
    int *ovf_count2;
    // composite order recorded by the forward for the backward's replay (hit_list == nullptr: off)
    unsigned *hit_list;       // [tiles][list_cap][256] record index of the k-th composited hit
    int list_cap;
    int *pix_cnt;             // [pixels] hits composited by the forward
};
cudaError_t launch_composite_fwd(const CompositeParams &p, int total_tiles, int tile, int chunk,
                                 int reorder_k, cudaStream_t s);
cudaError_t launch_composite_bwd(const CompositeParams &p, int total_tiles, int tile, int chunk,
                                 int reorder_k, cudaStream_t s);
cudaError_t launch_composite_fallback(const CompositeParams &p, int tile, bool bwd, cudaStream_t s);
cudaError_t launch_composite_replay(const CompositeParams &p, int total_tiles, int tile, cudaStream_t s);
// composite_loss.cu: the same with the loss channels (p.loss_sums set); the launchers above call them
cudaError_t launch_composite_loss(const CompositeParams &p, int total_tiles, int tile, int chunk, int reorder_k,
                                  bool bwd, cudaStream_t s);
cudaError_t launch_composite_fallback_loss(const CompositeParams &p, int tile, bool bwd, cudaStream_t s);
cudaError_t launch_composite_replay_loss(const CompositeParams &p, int total_tiles, int tile, cudaStream_t s);
// Opacity field at the exact depth of each pixel's ray over its recorded hits (forward), or its
// gradient into the record gradients (bwd).
cudaError_t launch_opacity_at_depth(const CompositeParams &p, int total_tiles, int tile, bool bwd, cudaStream_t s);
cudaError_t launch_grad_copies_zero(float4 *copies, const int *n_vis_dev, long long vis_cap, cudaStream_t s);
cudaError_t launch_grad_copies_reduce(const float4 *copies, const int *n_vis_dev, long long vis_cap, float4 *rgrad,
                                      cudaStream_t s);
// backward.cu
cudaError_t launch_preprocess_bwd(const SceneDev &sc, const CamSet *cams_dev, int n_views,
                                  float near_plane, const int *vflag, const int *vis_pos, int vis_cap,
                                  const float4 *rgrad, const sof_scene_grad &grad, cudaStream_t s);
// query.cu
cudaError_t launch_fill(float *p, long long n, float v, cudaStream_t s);
cudaError_t launch_point_append(const CamSet *cams_dev, int view, const float *pts, long long n_points,
                               float near_plane, int *seen, unsigned long long *cursor, unsigned *ptile,
                               unsigned *pkey, unsigned *pidx, unsigned *prank, int *tile_counts, cudaStream_t s);
cudaError_t launch_tile_blocks(const int *pcounts, int n_tiles, int *nb, cudaStream_t s);
cudaError_t launch_fill_lut(const int *nb, const int *bstart, int n_tiles, int2 *lut, cudaStream_t s);
// points_per_tile: the call's points over the view's tiles; from 1024 on (full point blocks) each
// thread walks two points, below it one.
cudaError_t launch_integrate(const CamSet *cams_dev, int view, const float4 *qrec, const unsigned long long *gpairs,
                             const int2 *granges, const unsigned long long *ppairs, const int2 *pranges,
                             const int2 *lut, const int *n_blocks, long long max_blocks, const float *pts,
                             float near_plane, float t_stop, bool level_set, float *opacity_out, DevStatus *status,
                             long long points_per_tile, cudaStream_t s);
// Level-set bisection: mid = (inside + outside) / 2 per edge; then inside or outside moves to mid
// as O(mid) > 0.5 or not.
cudaError_t launch_midpoints(const float *inside, const float *outside, long long n, float *mid, cudaStream_t s);
cudaError_t launch_bisect_update(float *inside, float *outside, const float *mid, const float *o_mid, long long n,
                                 cudaStream_t s);
}  // namespace sof
