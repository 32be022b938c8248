// C-ABI drivers (include/sof.h): argument checks, workspace layout, kernel orchestration.
// Every compute step runs in the kernels of this library; nothing here touches the data.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "sof_internal.cuh"

using namespace sof;

namespace sof {
static std::atomic<long long> g_launches{0};
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace sof

namespace {

// The first bytes of every layout: state that outlives one call (same address in every layout).
struct Persist {
    unsigned long long dropped;  // n_dropped summed over calls since sof_workspace_clear_dropped
};

struct Layout {
    size_t total = 0;
    Persist *persist = nullptr;
    CamSet *cams = nullptr;
    DevStatus *status = nullptr;
    int *total_dev = nullptr;
    // 64-bit counters: [0] binning items (the scan total of the tile counts), [1] pairs appended,
    // [2] pairs that pass (the reservation's counting pass)
    unsigned long long *big = nullptr;
    float4 *records = nullptr;
    float4 *aux = nullptr;
    int4 *rects = nullptr;
    int *counts = nullptr;          // [records] tiles of the rectangle (pair upper bound)
    long long *offsets = nullptr;   // [records] render: scan of vis_area (item offsets)
    int *vflag = nullptr, *vis_pos = nullptr, *vis_list = nullptr, *vis_area = nullptr;  // [records]
    void *scan_tmp = nullptr;
    unsigned *ptile = nullptr, *pkey = nullptr, *prec = nullptr;  // [pairs] unsorted (tile, key, record)
    unsigned long long *bucketed = nullptr;  // [pairs] grouped by tile: key bits << 32 | record
    // [pairs] the tiles' lists, each a sorted front and the rest; it takes the place of ptile and
    // pkey, which are dead once bucketed
    unsigned long long *pairs = nullptr;
    int *tile_counts = nullptr, *tile_offsets = nullptr, *tile_cursor = nullptr;  // [tiles]
    int2 *ranges = nullptr;
    int *prefix_end = nullptr, *tile_flag = nullptr;  // [tiles]
    int *block_first = nullptr;  // [pairs / 256 + 1] the record of each binning CTA's first item
    int *redo = nullptr;         // render: [1 + tiles] count, then the tiles the second pass redoes
    float4 *loss_sums = nullptr; // [pixels] the loss channels' per-pixel sums for the backward
    int *open_tiles = nullptr;                        // [2][tiles] tiles whose rest of the list is sorted
    float *prefix_key = nullptr;                      // [tiles]
    float4 *rgrad = nullptr;
    unsigned char *ovf_mask = nullptr;
    unsigned *ovf_list = nullptr, *ovf_list2 = nullptr;
    float4 *grad_copies = nullptr; // [records][kGradCopies][6] backward accumulators
    unsigned *hit_list = nullptr;  // [tiles][list_cap][256] composite order for the backward
    int *pix_cnt = nullptr;        // [pixels] hits composited per pixel
};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

// Bump layout of one render or query call; with base == nullptr only sizes are computed. items: the
// binning-item capacity (block table), -1 = pairs.
Layout make_layout(char *base, long long n_rec, long long pairs, int tiles, bool rgrad, long long pixels = 0,
                   int list_cap = 0, long long vis_cap = 0, int tile = 16, long long items = -1) {
    if (items < 0) items = pairs;
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += al(bytes);
        return p;
    };
    L.persist = reinterpret_cast<Persist *>(take(sizeof(Persist)));
    L.cams = reinterpret_cast<CamSet *>(take(sizeof(CamSet)));
    L.status = reinterpret_cast<DevStatus *>(take(sizeof(DevStatus)));
    L.total_dev = reinterpret_cast<int *>(take(sizeof(int) * 8));
    L.big = reinterpret_cast<unsigned long long *>(take(sizeof(unsigned long long) * 8));
    L.records = reinterpret_cast<float4 *>(take((size_t)n_rec * kRecF4 * sizeof(float4)));
    L.aux = reinterpret_cast<float4 *>(take((size_t)n_rec * sizeof(float4)));
    L.rects = reinterpret_cast<int4 *>(take((size_t)n_rec * sizeof(int4)));
    L.counts = reinterpret_cast<int *>(take((size_t)n_rec * sizeof(int)));
    L.offsets = reinterpret_cast<long long *>(take((size_t)n_rec * sizeof(long long)));
    L.vflag = reinterpret_cast<int *>(take((size_t)n_rec * sizeof(int)));
    L.vis_pos = reinterpret_cast<int *>(take((size_t)n_rec * sizeof(int)));
    L.vis_list = reinterpret_cast<int *>(take((size_t)n_rec * sizeof(int)));
    L.vis_area = reinterpret_cast<int *>(take((size_t)n_rec * sizeof(int)));
    L.scan_tmp = take(scan_temp_bytes(std::max<long long>(n_rec, tiles)));
    char *tk = take((size_t)pairs * 8);
    L.ptile = reinterpret_cast<unsigned *>(tk);
    L.pkey = tk ? reinterpret_cast<unsigned *>(tk + (size_t)pairs * 4) : nullptr;
    L.pairs = reinterpret_cast<unsigned long long *>(tk);
    L.prec = reinterpret_cast<unsigned *>(take((size_t)pairs * 4));
    L.bucketed = reinterpret_cast<unsigned long long *>(take((size_t)pairs * 8));
    L.prefix_end = reinterpret_cast<int *>(take((size_t)tiles * sizeof(int)));
    L.tile_flag = reinterpret_cast<int *>(take((size_t)tiles * sizeof(int)));
    L.open_tiles = reinterpret_cast<int *>(take((size_t)tiles * 2 * sizeof(int)));
    L.redo = reinterpret_cast<int *>(take((size_t)(tiles + 1) * sizeof(int)));
    L.prefix_key = reinterpret_cast<float *>(take((size_t)tiles * sizeof(float)));
    L.block_first = reinterpret_cast<int *>(take(((size_t)items / 256 + 1) * sizeof(int)));
    L.loss_sums = reinterpret_cast<float4 *>(take((size_t)pixels * sizeof(float4)));
    L.tile_counts = reinterpret_cast<int *>(take((size_t)tiles * sizeof(int)));
    L.tile_offsets = reinterpret_cast<int *>(take((size_t)tiles * sizeof(int)));
    L.tile_cursor = reinterpret_cast<int *>(take((size_t)tiles * sizeof(int)));
    L.ranges = reinterpret_cast<int2 *>(take((size_t)tiles * sizeof(int2)));
    if (rgrad) L.rgrad = reinterpret_cast<float4 *>(take((size_t)vis_cap * kGradF4 * sizeof(float4)));
    L.ovf_mask = reinterpret_cast<unsigned char *>(take((size_t)pixels));
    L.ovf_list = reinterpret_cast<unsigned *>(take((size_t)pixels * sizeof(unsigned)));
    L.ovf_list2 = reinterpret_cast<unsigned *>(take((size_t)pixels * sizeof(unsigned)));
    if (rgrad)
        L.grad_copies = reinterpret_cast<float4 *>(take((size_t)vis_cap * kGradCopies * kGradF4 * sizeof(float4)));
    if (list_cap > 0) {
        L.hit_list = reinterpret_cast<unsigned *>(take((size_t)tiles * list_cap * tile * tile * sizeof(unsigned)));
        L.pix_cnt = reinterpret_cast<int *>(take((size_t)pixels * sizeof(int)));
    }
    L.total = off;
    return L;
}

}  // namespace

struct sof_workspace {
    char *base = nullptr;
    size_t bytes = 0;
    size_t required = 0;
    char err[512] = {0};
    CamSet cams;
    Layout L;
    // state a forward leaves for its backward
    bool fwd_valid = false;
    long long fwd_n = -1;
    int fwd_views = 0;
    int tile = 16, chunk = 64, k = 16, list_cap = 0;
    bool approx = false, losses = false;
    long long vis_cap = 0;   // visible-record capacity of the last forward's layout
    long long vis_hint = 0;  // visible records seen by the last synchronous forward
    long long item_hint = 0; // binning items counted by sof_workspace_reserve (grows only)
    // resident query state left by sof_query_prepare (valid until the workspace is rebound or a
    // call other than a prepared query lays out its scratch over it)
    struct Prepared {
        bool valid = false;
        long long n = 0;
        int n_views = 0, tile = 16, max_tiles = 0;
        float near_plane = 0.f;
        CamSet cams;                       // as built for the views (compared by later queries)
        std::vector<long long> pair_off;   // [views + 1] each view's first sorted pair
        size_t records = 0, pairs = 0, ranges = 0, cams_dev = 0, end = 0;  // byte offsets
    } prep;
    float near_plane = 0.2f, t_stop = 1e-4f;
    bool persist_stale = true;  // the bound memory's persistent counters are not cleared yet
    CamSet fwd_cams;       // cameras of the last forward (compared by its backward)
    sof_render_out fwd_out = {};  // output pointers of the last forward (idem)
    cudaStream_t last_stream = nullptr;
    long long last_point_views = 0;
    // phase timing (sof_workspace_set_timing): event pairs recorded since the last read
    bool timing = false;
    struct Timed {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t event() {
        cudaEvent_t e = nullptr;
        if (!pool.empty()) {
            e = pool.back();
            pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
        }
        return e;
    }
    ~sof_workspace() {
        for (auto &t : timed) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

namespace {
// Records an event pair around the launches of one phase on the call's stream while timing is on.
struct PhaseTimer {
    sof_workspace *ws;
    int phase;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    PhaseTimer(sof_workspace *w, int ph, cudaStream_t st) : ws(w), phase(ph), s(st) {
        if (ws->timing && (a = ws->event())) cudaEventRecord(a, s);
    }
    ~PhaseTimer() {
        if (!a) return;
        cudaEvent_t b = ws->event();
        if (!b) {
            ws->pool.push_back(a);
            return;
        }
        cudaEventRecord(b, s);
        ws->timed.push_back({phase, a, b});
    }
};
}  // namespace
#define SOF_PHASE(ws, ph, s) PhaseTimer phase_timer_##ph((ws), (ph), (s))

namespace {

int cuda_fail(sof_workspace *ws, cudaError_t e, const char *what) {
    if (ws) snprintf(ws->err, sizeof(ws->err), "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return SOF_ERR_CUDA;
}

#define SOF_CUDA(ws, call)                                     \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(ws, e_, #call); \
    } while (0)

int check_device(sof_workspace *ws) {
    static int cached = 0;  // 1 ok, -1 bad
    if (cached == 1) return SOF_OK;
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        if (ws) snprintf(ws->err, sizeof(ws->err), "no CUDA device");
        return SOF_ERR_NO_DEVICE;
    }
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (major != 10 || minor != 3) {
        if (ws) snprintf(ws->err, sizeof(ws->err), "device %d has compute capability %d.%d; this library is built for sm_103a",
                         dev, major, minor);
        return SOF_ERR_NO_DEVICE;
    }
    cached = 1;
    return SOF_OK;
}

int validate_scene(const sof_scene *sc, bool need_sh) {
    if (!sc || sc->n < 0 || sc->sh_degree < 0 || sc->sh_degree > SOF_MAX_SH_DEGREE) return SOF_ERR_INVALID_ARG;
    if (sc->n > 0 && (!sc->means || !sc->log_scales || !sc->quats || !sc->opacity_logits)) return SOF_ERR_INVALID_ARG;
    if (sc->n > 0 && need_sh && !sc->sh) return SOF_ERR_INVALID_ARG;
    if (sc->n > 0 && ((uintptr_t)sc->quats & 15)) return SOF_ERR_INVALID_ARG;  // read as float4
    if (sc->n >= (1ll << 31) / SOF_MAX_VIEWS) return SOF_ERR_INVALID_ARG;
    return SOF_OK;
}

// FP64 camera preparation from the FP32 inputs; tiles laid out view after view.
int build_cams(const sof_camera *cams, int n_views, int tile, float near_plane, CamSet *out) {
    if (!cams || n_views < 1 || n_views > SOF_MAX_VIEWS) return SOF_ERR_INVALID_ARG;
    out->n_views = n_views;
    out->tile = tile;
    long long tbase = 0, pbase = 0;
    for (int v = 0; v < n_views; ++v) {
        const sof_camera &c = cams[v];
        DevCam &d = out->cam[v];
        memset(&d, 0, sizeof(d));
        if (c.width <= 0 || c.height <= 0 || c.width > 65536 || c.height > 65536) return SOF_ERR_INVALID_ARG;
        if (!(c.fx > 0.f) || !(c.fy > 0.f) || !isfinite(c.cx) || !isfinite(c.cy) || !isfinite(c.fx) || !isfinite(c.fy))
            return SOF_ERR_INVALID_ARG;
        for (int i = 0; i < 12; ++i)
            if (!isfinite(c.world_to_cam[i])) return SOF_ERR_INVALID_ARG;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) {
                d.R[3 * i + j] = (double)c.world_to_cam[4 * i + j];
                d.Rf[3 * i + j] = c.world_to_cam[4 * i + j];
            }
            d.t[i] = (double)c.world_to_cam[4 * i + 3];
            d.tf[i] = c.world_to_cam[4 * i + 3];
        }
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int i = 0; i < 3; ++i) acc -= d.R[3 * i + j] * d.t[i];
            d.cf[j] = (float)acc;
        }
        d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
        d.rfx = 1.0 / (double)c.fx;
        d.rfy = 1.0 / (double)c.fy;
        d.W = c.width; d.H = c.height;
        d.tiles_x = (c.width + tile - 1) / tile;
        d.tiles_y = (c.height + tile - 1) / tile;
        double umax = std::max(fabs(0.5 - (double)c.cx), fabs((double)c.width - 0.5 - (double)c.cx)) / c.fx;
        double vmax = std::max(fabs(0.5 - (double)c.cy), fabs((double)c.height - 0.5 - (double)c.cy)) / c.fy;
        d.zclip = (float)(near_plane / sqrt(1.0 + umax * umax + vmax * vmax) * (1.0 - 1e-5));
        d.tile_base = (int)tbase;
        d.pix_base = pbase;
        tbase += (long long)d.tiles_x * d.tiles_y;
        pbase += (long long)c.width * c.height;
        // the composite's overflow lists code (tile << bits | thread), bits = log2(tile * tile)
        const int tid_bits = tile == 8 ? 6 : (tile == 16 ? 8 : 10);
        if (tbase >= (1ll << 31) || (tbase << tid_bits) > (1ll << 32)) return SOF_ERR_INVALID_ARG;
    }
    out->total_tiles = (int)tbase;
    return SOF_OK;
}

size_t cams_bytes(int n_views) { return offsetof(CamSet, cam) + (size_t)n_views * sizeof(DevCam); }

long long total_pixels(const CamSet &cs) {
    long long p = 0;
    for (int v = 0; v < cs.n_views; ++v) p += (long long)cs.cam[v].W * cs.cam[v].H;
    return p;
}

int tile_bits(int total_tiles) {
    int b = 0;
    while ((1ll << b) < total_tiles) ++b;
    return b;
}

constexpr int kSecondPassK = 64;  // buffer of the composite's second pass over overflowed pixels

// Binning-item capacity of a stream-ordered render sized by sof_workspace_reserve: the items it
// counted with 1/16 slack (-1 without a reservation: as many items as pairs).
long long reserved_items(long long hint) { return hint > 0 ? hint + hint / 16 + 1024 : -1; }

// Visible-record capacity of a render layout: the last synchronous call's count with 25% slack,
// at least 65536 (or all records).
long long default_vis_cap(long long n_rec, long long hint) {
    return std::min<long long>(n_rec, std::max<long long>(65536, hint + hint / 4));
}

constexpr int kDefaultSortPrefix = 256;

int resolve_opts(const sof_render_opts *o, int *tile, int *chunk, int *k, int *list_cap, int *prefix = nullptr) {
    if (prefix) *prefix = o->sort_prefix == 0 ? kDefaultSortPrefix : (o->sort_prefix < 0 ? 0 : o->sort_prefix);
    if (o->sort_prefix < -1) return SOF_ERR_INVALID_ARG;
    *tile = o->tile == 0 ? 16 : o->tile;
    *list_cap = o->replay_cap == 0 ? 256 : (o->replay_cap < 0 ? 0 : o->replay_cap);
    if (o->replay_cap < -1 || o->replay_cap > 4096) return SOF_ERR_INVALID_ARG;
    *chunk = o->chunk == 0 ? 64 : o->chunk;
    *k = o->reorder_k == 0 ? 16 : o->reorder_k;
    if (*tile != 8 && *tile != 16 && *tile != 32) return SOF_ERR_INVALID_ARG;
    if (*chunk != 32 && *chunk != 64 && *chunk != 128) return SOF_ERR_INVALID_ARG;
    if (*k != 8 && *k != 16 && *k != 32) return SOF_ERR_INVALID_ARG;
    if (*chunk == 128 && *k != 16) return SOF_ERR_INVALID_ARG;
    // instantiated at tiles of 8: chunk 64 with buffers of 16 or 32; of 32: chunk 64 with 8 or 16
    if (*tile == 8 && (*chunk != 64 || *k == 8)) return SOF_ERR_INVALID_ARG;
    if (*tile == 32 && (*chunk != 64 || *k == 32)) return SOF_ERR_INVALID_ARG;
    if (!(o->near_plane >= 0.f) || !(o->t_stop >= 0.f) || !(o->t_stop < 1.f)) return SOF_ERR_INVALID_ARG;
    return SOF_OK;
}

// Largest pair capacity whose layout fits in `bytes` (items: the item capacity, -1 = the pairs').
long long fit_pairs(size_t bytes, long long n_rec, int tiles, bool rgrad, long long pixels, int list_cap,
                    long long vis_cap, int tile, long long items = -1) {
    auto need = [&](long long pairs) {
        return make_layout(nullptr, n_rec, pairs, tiles, rgrad, pixels, list_cap, vis_cap, tile, items).total;
    };
    if (need(0) > bytes) return -1;
    long long lo = 0, hi = 1;
    while (need(hi) <= bytes && hi < (1ll << 31)) hi *= 2;
    while (hi - lo > 1) {
        long long mid = (lo + hi) / 2;
        if (need(mid) <= bytes) lo = mid;
        else hi = mid;
    }
    return std::min<long long>(lo, (1ll << 31) - 1);
}

}  // namespace

extern "C" {

int sof_version(void) { return 1; }

const char *sof_error_string(int code) {
    switch (code) {
        case SOF_OK: return "ok";
        case SOF_WARN_INEXACT: return "warning: some pixels could not keep exact depth order";
        case SOF_ERR_INVALID_ARG: return "invalid argument";
        case SOF_ERR_CUDA: return "CUDA error";
        case SOF_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
        case SOF_ERR_NOT_IMPLEMENTED: return "not implemented";
        case SOF_ERR_NO_DEVICE: return "no sm_103 CUDA device";
        case SOF_ERR_STATE: return "backward without a matching forward on this workspace";
        default: return "unknown status";
    }
}

const char *sof_last_cuda_error(const sof_workspace *ws) { return ws ? ws->err : ""; }

int sof_workspace_create(sof_workspace **ws) {
    if (!ws) return SOF_ERR_INVALID_ARG;
    *ws = new sof_workspace();
    return SOF_OK;
}

int sof_workspace_destroy(sof_workspace *ws) {
    delete ws;
    return SOF_OK;
}

int sof_workspace_bind(sof_workspace *ws, void *device_ptr, size_t bytes) {
    if (!ws || (bytes > 0 && !device_ptr) || ((uintptr_t)device_ptr & 255)) return SOF_ERR_INVALID_ARG;
    ws->base = reinterpret_cast<char *>(device_ptr);
    ws->bytes = bytes;
    ws->fwd_valid = false;
    ws->persist_stale = true;  // cleared on the stream by the next call that lays it out
    ws->prep.valid = false;
    return SOF_OK;
}

int sof_workspace_required(const sof_workspace *ws, size_t *bytes) {
    if (!ws || !bytes) return SOF_ERR_INVALID_ARG;
    *bytes = ws->required;
    return SOF_OK;
}

int sof_workspace_clear_dropped(sof_workspace *ws, void *stream) {
    if (!ws) return SOF_ERR_INVALID_ARG;
    if (!ws->base) return SOF_OK;
    SOF_CUDA(ws, cudaMemsetAsync(ws->base, 0, sizeof(Persist), reinterpret_cast<cudaStream_t>(stream)));
    ws->persist_stale = false;
    return SOF_OK;
}

}  // extern "C"

namespace sof {
bool workspace_timing(const sof_workspace *ws) { return ws->timing; }
size_t workspace_bytes(const sof_workspace *ws) { return ws->base ? ws->bytes : 0; }
void workspace_set_required(sof_workspace *ws, size_t bytes) { ws->required = bytes; }
void workspace_note(sof_workspace *ws, const char *msg) { snprintf(ws->err, sizeof(ws->err), "%s", msg); }
}  // namespace sof

extern "C" {

int sof_workspace_set_timing(sof_workspace *ws, int enable) {
    if (!ws) return SOF_ERR_INVALID_ARG;
    ws->timing = enable != 0;
    return SOF_OK;
}

int sof_workspace_timing(sof_workspace *ws, double *ms, int64_t *launches) {
    if (!ws || !ms || !launches) return SOF_ERR_INVALID_ARG;
    for (int i = 0; i < SOF_N_PHASES; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    int rc = SOF_OK;
    for (auto &t : ws->timed) {
        float el = 0.f;
        if (cudaEventSynchronize(t.b) != cudaSuccess || cudaEventElapsedTime(&el, t.a, t.b) != cudaSuccess)
            rc = SOF_ERR_CUDA;
        if (t.phase >= 0 && t.phase < SOF_N_PHASES) {
            ms[t.phase] += el;
            launches[t.phase] += 1;
        }
        ws->pool.push_back(t.a);
        ws->pool.push_back(t.b);
    }
    ws->timed.clear();
    return rc;
}

int sof_render_workspace_size(const sof_scene *scene, const sof_camera *cams, int n_views,
                              const sof_render_opts *opts, int64_t pair_capacity, size_t *bytes) {
    if (!bytes || !opts || pair_capacity < 0) return SOF_ERR_INVALID_ARG;
    int rc = validate_scene(scene, true);
    if (rc) return rc;
    int tile, chunk, k, list_cap;
    if ((rc = resolve_opts(opts, &tile, &chunk, &k, &list_cap))) return rc;
    thread_local CamSet tmp;
    if ((rc = build_cams(cams, n_views, tile, opts->near_plane, &tmp))) return rc;
    const long long n_rec = scene->n * n_views;
    *bytes = make_layout(nullptr, n_rec, pair_capacity, tmp.total_tiles, true, total_pixels(tmp), list_cap,
                         default_vis_cap(n_rec, 0), tile).total;
    return SOF_OK;
}

int sof_workspace_stats(const sof_workspace *ws, sof_stats *st) {
    if (!ws || !st) return SOF_ERR_INVALID_ARG;
    memset(st, 0, sizeof(*st));
    if (!ws->base || !ws->L.status) return SOF_OK;
    DevStatus ds;
    if (cudaStreamSynchronize(ws->last_stream) != cudaSuccess) return SOF_ERR_CUDA;
    if (cudaMemcpy(&ds, ws->L.status, sizeof(ds), cudaMemcpyDeviceToHost) != cudaSuccess) return SOF_ERR_CUDA;
    unsigned long long c[kCntFields] = {0};
    for (int i = 0; i < kCntShards; ++i)
        for (int f = 0; f < kCntFields; ++f) c[f] += ds.cnt[i][f];
    st->n_pairs = (int64_t)ds.n_pairs;
    st->n_visible = (int64_t)c[kCntVisible];
    st->inexact_pixels = (int64_t)ds.inexact_pixels;
    st->nonfinite = (int64_t)ds.nonfinite;
    st->n_point_views = (int64_t)c[kCntPointViews];
    st->n_tests = (int64_t)c[kCntTests];
    st->n_hits = (int64_t)c[kCntHits];
    st->n_composited = (int64_t)c[kCntComposited];
    st->n_forced = (int64_t)ds.n_forced;
    st->n_below_key = (int64_t)ds.n_below_key;
    st->n_unsorted = (int64_t)ds.n_unsorted;
    st->n_replayed = (int64_t)c[kCntReplayed];
    st->n_open = (int64_t)ds.n_open;
    st->n_read = (int64_t)c[kCntRead];
    // render: summed over the forwards since sof_workspace_clear_dropped; query: this call's
    unsigned long long dropped = ds.n_dropped;
    if (ws->L.persist &&
        cudaMemcpy(&dropped, &ws->L.persist->dropped, sizeof(dropped), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SOF_ERR_CUDA;
    st->n_dropped = (int64_t)dropped;
    return SOF_OK;
}

int64_t sof_kernel_launches(void) { return (int64_t)sof::g_launches.load(); }

}  // extern "C"

namespace {
// How a forward treats the capacities of its workspace.
enum FwdMode {
    kFwdStream,   // stream-ordered (the default): capacities from the bound workspace, excess dropped
    kFwdChecked,  // SOF_FLAG_CHECKED: one host round trip; a too-small workspace is an error
    kFwdReserve   // sof_workspace_reserve: stop after the pair bound and report the size needed
};

// The forward render. for_backward: lay out the gradient copies and replay lists a following
// sof_render_bwd needs (false only for the forward-only no-allocation entry point).
int render_fwd_impl(const sof_scene *scene, const sof_camera *cams, int n_views, const sof_render_opts *opts,
                    const sof_render_out *out, sof_workspace *ws, void *stream, FwdMode mode, bool for_backward,
                    size_t *reserve_bytes) {
    if (!ws || !opts || (!out && mode != kFwdReserve)) return SOF_ERR_INVALID_ARG;
    ws->fwd_valid = false;
    ws->prep.valid = false;  // the render's layout starts at the front of the workspace
    ws->required = 0;
    int rc = validate_scene(scene, true);
    if (rc) return rc;
    if (opts->flags & ~(SOF_FLAG_MEDIAN_DEPTH | SOF_FLAG_ASYNC | SOF_FLAG_APPROX_ORDER | SOF_FLAG_CHECKED))
        return SOF_ERR_INVALID_ARG;
    if (mode != kFwdReserve &&
        (!out->color || !out->depth || !out->exact_depth || !out->normal || !out->opacity || !out->n_contrib))
        return SOF_ERR_INVALID_ARG;
    int tile, chunk, k, list_cap, prefix;
    if ((rc = resolve_opts(opts, &tile, &chunk, &k, &list_cap, &prefix))) return rc;
    if (!for_backward) list_cap = 0;
    const bool losses = mode != kFwdReserve && (out->distortion || out->extent);
    // the opacity at the exact depth walks the recorded hits
    if (mode != kFwdReserve && out->opacity_at_depth && list_cap <= 0) return SOF_ERR_INVALID_ARG;
    if ((rc = check_device(ws))) return rc;
    if ((rc = build_cams(cams, n_views, tile, opts->near_plane, &ws->cams))) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ws->last_stream = s;
    const long long n = scene->n, n_rec = n * n_views;
    const int tiles = ws->cams.total_tiles;
    const long long npx = total_pixels(ws->cams);
    const bool async = mode == kFwdStream;
    // the reservation lays out only what precedes the pair bound, and counts every visible record
    const long long vis_cap = mode == kFwdReserve ? n_rec : default_vis_cap(n_rec, ws->vis_hint);
    // binning items: a stream-ordered forward after a reservation has its own item capacity (the
    // pairs that pass are far fewer than the items tested); otherwise one per pair of capacity
    const long long item_cap = mode == kFwdStream ? reserved_items(ws->item_hint) : -1;
    long long cap = mode == kFwdReserve ? 0
                                        : fit_pairs(ws->bytes, n_rec, tiles, for_backward, npx, list_cap, vis_cap, tile,
                                                    item_cap);
    const size_t reserve_total = make_layout(nullptr, n_rec, 0, tiles, false, 0, 0, 0, tile).total;
    if (cap < 0 || !ws->base || (mode == kFwdReserve && reserve_total > ws->bytes)) {
        ws->required = mode == kFwdReserve ? reserve_total
                                           : make_layout(nullptr, n_rec, std::max<long long>(n_rec * 4, 1024), tiles,
                                                         for_backward, npx, list_cap, vis_cap, tile).total;
        return SOF_ERR_WORKSPACE_TOO_SMALL;
    }
    Layout L = mode == kFwdReserve
                   ? make_layout(ws->base, n_rec, 0, tiles, false, 0, 0, 0, tile)
                   : make_layout(ws->base, n_rec, cap, tiles, for_backward, npx, list_cap, vis_cap, tile, item_cap);
    const long long items_max = item_cap < 0 ? cap : item_cap;  // the block table's capacity
    ws->L = L;
    ws->vis_cap = vis_cap;
    SceneDev sc{scene->means, scene->log_scales, scene->quats, scene->opacity_logits, scene->sh, n, scene->sh_degree};

    SOF_CUDA(ws, launch_set_cams(ws->cams, L.cams, s));
    SOF_CUDA(ws, cudaMemsetAsync(L.status, 0, sizeof(DevStatus), s));
    // a checked call drops nothing; a stream-ordered one starts the count on memory just bound
    if (!async || ws->persist_stale) SOF_CUDA(ws, cudaMemsetAsync(L.persist, 0, sizeof(Persist), s));
    ws->persist_stale = false;
    // [0] pair upper bound, [1] pairs appended, [2] pairs bucketed, [3] overflowed pixels,
    // [4] records with tiles, [5] second-pass overflows, [6] [7] open tiles of the two passes
    SOF_CUDA(ws, cudaMemsetAsync(L.total_dev, 0, 8 * sizeof(int), s));
    SOF_CUDA(ws, cudaMemsetAsync(L.big, 0, 8 * sizeof(unsigned long long), s));
    SOF_CUDA(ws, cudaMemsetAsync(L.vis_area, 0, (size_t)n_rec * sizeof(int), s));
    if (mode != kFwdReserve) {
        SOF_CUDA(ws, cudaMemsetAsync(L.tile_counts, 0, (size_t)tiles * sizeof(int), s));
        SOF_CUDA(ws, cudaMemsetAsync(L.redo, 0, sizeof(int), s));
    }
    {
        SOF_PHASE(ws, SOF_PHASE_PREPROCESS, s);
        SOF_CUDA(ws, launch_preprocess(sc, L.cams, ws->cams, opts->near_plane, false, L.records, L.aux, L.rects,
                                       L.status, s));
    }
    {
        SOF_PHASE(ws, SOF_PHASE_BIN_COUNT, s);
        SOF_CUDA(ws, launch_rect_area(L.aux, L.rects, n_rec, L.counts, L.vflag, s));
    }
    {
        SOF_PHASE(ws, SOF_PHASE_SCAN, s);
        SOF_CUDA(ws, launch_exclusive_scan(L.vflag, L.vis_pos, n_rec, L.scan_tmp, L.total_dev + 4, s));
        SOF_CUDA(ws, launch_compact_visible(L.counts, L.vflag, L.vis_pos, n_rec, L.vis_list, L.vis_area, vis_cap,
                                            &L.status->n_dropped, s));
        SOF_CUDA(ws, launch_exclusive_scan64(L.vis_area, L.offsets, n_rec, L.scan_tmp,
                                             reinterpret_cast<long long *>(L.big), s));
    }
    long long items = items_max;  // without the round trip: the item capacity
    if (!async) {
        // the checked forward's (and the reservation's) host round trip: the binning items and the
        // visible records decide whether the workspace is large enough
        int hv[5] = {0, 0, 0, 0, 0};
        long long n_items = 0;
        SOF_CUDA(ws, cudaMemcpyAsync(hv, L.total_dev, sizeof(hv), cudaMemcpyDeviceToHost, s));
        SOF_CUDA(ws, cudaMemcpyAsync(&n_items, L.big, sizeof(n_items), cudaMemcpyDeviceToHost, s));
        SOF_CUDA(ws, cudaStreamSynchronize(s));
        const int n_vis = hv[4];
        if (n_items < 0 || n_vis < 0) return SOF_ERR_CUDA;
        ws->vis_hint = std::max<long long>(ws->vis_hint, n_vis);  // grows only: calls of a step share it
        if (mode == kFwdReserve) {
            // count the pairs that pass the tile test (nothing is written), then size the
            // stream-ordered forward: those pairs with 1/8 slack, the items with 1/16
            {
                SOF_PHASE(ws, SOF_PHASE_BIN_EMIT, s);
                SOF_CUDA(ws, launch_bin_append(L.cams, n, L.records, L.aux, L.rects, L.vis_list, L.offsets,
                                               L.total_dev + 4, reinterpret_cast<const long long *>(L.big), n_items,
                                               false, opts->near_plane, 0, L.big + 2, nullptr, nullptr, nullptr,
                                               nullptr, nullptr, s, nullptr));
            }
            unsigned long long passing = 0;
            SOF_CUDA(ws, cudaMemcpyAsync(&passing, L.big + 2, sizeof(passing), cudaMemcpyDeviceToHost, s));
            SOF_CUDA(ws, cudaStreamSynchronize(s));
            if (passing >= (unsigned long long)INT32_MAX - (passing >> 3) - 4096) {
                snprintf(ws->err, sizeof(ws->err),
                         "%llu (Gaussian, tile) pairs exceed one call's 32-bit pair indexing: render fewer views "
                         "per call", passing);
                return SOF_ERR_INVALID_ARG;
            }
            ws->item_hint = std::max<long long>(ws->item_hint, n_items);
            const long long pairs = (long long)passing + (long long)(passing >> 3) + 1024;
            *reserve_bytes = make_layout(nullptr, n_rec, pairs, tiles, for_backward, npx, list_cap,
                                         default_vis_cap(n_rec, ws->vis_hint), tile,
                                         reserved_items(ws->item_hint)).total;
            return SOF_OK;
        }
        // checked: one pair of capacity per item (the pair indices are 32-bit)
        if (n_items > (long long)INT32_MAX - 1024) {
            snprintf(ws->err, sizeof(ws->err),
                     "%lld (Gaussian, tile) candidate pairs exceed a checked call's 32-bit indexing: size the "
                     "workspace with sof_workspace_reserve and render stream-ordered, or render fewer views per "
                     "call", n_items);
            return SOF_ERR_INVALID_ARG;
        }
        if (n_items > cap || n_vis > vis_cap) {
            ws->required = make_layout(nullptr, n_rec, std::max<long long>(n_items + n_items / 8 + 1024, cap), tiles,
                                       for_backward, npx, list_cap, default_vis_cap(n_rec, ws->vis_hint), tile).total;
            return SOF_ERR_WORKSPACE_TOO_SMALL;
        }
        items = n_items;
    }
    {
        SOF_PHASE(ws, SOF_PHASE_BIN_EMIT, s);
        const long long *n_items_dev = reinterpret_cast<const long long *>(L.big);
        SOF_CUDA(ws, launch_block_first(L.offsets, L.total_dev + 4, n_items_dev, n_rec, items, L.block_first, s));
        SOF_CUDA(ws, launch_bin_append(L.cams, n, L.records, L.aux, L.rects, L.vis_list, L.offsets, L.total_dev + 4,
                                       n_items_dev, items, false, opts->near_plane, cap, L.big + 1, L.ptile,
                                       L.pkey, L.prec, L.tile_counts, &L.status->n_dropped, s, L.block_first));
    }
    const FrontSort fs{L.pairs, prefix, L.prefix_end, L.prefix_key, L.tile_flag};
    {
        SOF_PHASE(ws, SOF_PHASE_SORT, s);
        SOF_CUDA(ws, launch_exclusive_scan(L.tile_counts, L.tile_offsets, tiles, L.scan_tmp, L.total_dev + 2, s));
        SOF_CUDA(ws, launch_tile_buckets(L.ptile, L.pkey, L.prec, L.big + 1, cap, L.tile_counts,
                                         L.tile_offsets, tiles, L.ranges, L.tile_cursor, L.bucketed,
                                         &L.status->n_pairs, s, &fs));
    }
    CompositeParams p;
    memset(&p, 0, sizeof(p));
    p.cams = L.cams;
    p.records = L.records;
    p.pairs = L.pairs;
    p.ranges = L.ranges;
    p.prefix_end = L.prefix_end;
    p.prefix_key = L.prefix_key;
    p.tile_flag = L.tile_flag;
    p.open_tiles[0] = L.open_tiles;
    p.open_tiles[1] = L.open_tiles + tiles;
    p.open_count[0] = L.total_dev + 6;
    p.open_count[1] = L.total_dev + 7;
    p.redo_count = L.redo;
    p.redo_tiles = L.redo + 1;
    p.near_plane = opts->near_plane;
    p.t_stop = opts->t_stop;
    for (int c = 0; c < 3; ++c) p.bg[c] = opts->bg[c];
    p.color = out->color;
    p.depth = out->depth;
    p.exact_depth = out->exact_depth;
    p.median_depth = (opts->flags & SOF_FLAG_MEDIAN_DEPTH) ? out->median_depth : nullptr;
    p.normal = out->normal;
    p.opacity = out->opacity;
    p.n_contrib = out->n_contrib;
    p.status = L.status;
    p.ovf_mask = L.ovf_mask;
    p.ovf_list = L.ovf_list;
    p.ovf_count = L.total_dev + 3;
    p.ovf_list2 = L.ovf_list2;
    p.ovf_count2 = L.total_dev + 5;
    p.hit_list = L.hit_list;
    p.list_cap = list_cap;
    p.pix_cnt = L.pix_cnt;
    p.approx = (opts->flags & SOF_FLAG_APPROX_ORDER) != 0;
    if (losses) {
        p.distortion = out->distortion;
        p.extent = out->extent;
        p.loss_sums = L.loss_sums;
    }
    {
        SOF_PHASE(ws, SOF_PHASE_COMPOSITE, s);
        SOF_CUDA(ws, launch_composite_fwd(p, tiles, tile, chunk, k, s));
    }
    {
        SOF_PHASE(ws, SOF_PHASE_FALLBACK, s);
        // the rest of the lists that the second pass and then the fallback read
        if (prefix > 0)
            SOF_CUDA(ws, launch_tail_sort(L.ranges, L.prefix_end, p.open_tiles[0], p.open_count[0], L.pairs, s));
        p.pass = 1;
        // tiles of 32 pixels have no second pass: their first pass lists its pixels for the fallback
        if (tile != 32) SOF_CUDA(ws, launch_composite_fwd(p, tiles, tile, chunk, kSecondPassK, s));
        if (prefix > 0)
            SOF_CUDA(ws, launch_tail_sort(L.ranges, L.prefix_end, p.open_tiles[1], p.open_count[1], L.pairs, s));
        SOF_CUDA(ws, launch_composite_fallback(p, tile, false, s));
    }
    if (out->opacity_at_depth) {
        p.opa = out->opacity_at_depth;
        SOF_CUDA(ws, launch_opacity_at_depth(p, tiles, tile, false, s));
    }
    SOF_CUDA(ws, launch_add_u64(&L.status->n_dropped, &L.persist->dropped, s));
    ws->fwd_n = n;
    ws->fwd_views = n_views;
    ws->tile = tile;
    ws->chunk = chunk;
    ws->k = k;
    ws->list_cap = list_cap;
    ws->approx = (opts->flags & SOF_FLAG_APPROX_ORDER) != 0;
    ws->losses = losses;
    ws->near_plane = opts->near_plane;
    ws->t_stop = opts->t_stop;
    ws->fwd_out = *out;
    ws->fwd_cams = ws->cams;
    ws->fwd_valid = for_backward;
    return SOF_OK;
}
}  // namespace

extern "C" {

int sof_render_fwd(const sof_scene *scene, const sof_camera *cams, int n_views, const sof_render_opts *opts,
                   const sof_render_out *out, sof_workspace *ws, void *stream) {
    const FwdMode mode = (opts && (opts->flags & SOF_FLAG_CHECKED)) ? kFwdChecked : kFwdStream;
    return render_fwd_impl(scene, cams, n_views, opts, out, ws, stream, mode, true, nullptr);
}

int sof_workspace_reserve(sof_workspace *ws, const sof_scene *scene, const sof_camera *cams, int n_views,
                          const sof_render_opts *opts, void *stream, size_t *bytes) {
    if (!bytes) return SOF_ERR_INVALID_ARG;
    *bytes = 0;
    return render_fwd_impl(scene, cams, n_views, opts, nullptr, ws, stream, kFwdReserve, true, bytes);
}

int sof_render_bwd(const sof_scene *scene, const sof_camera *cams, int n_views, const sof_render_opts *opts,
                   const sof_render_out *fwd, const sof_render_grad_in *gin, const sof_scene_grad *grad,
                   sof_workspace *ws, void *stream) {
    if (!ws || !opts || !fwd || !gin || !grad) return SOF_ERR_INVALID_ARG;
    int rc = validate_scene(scene, true);
    if (rc) return rc;
    if (!fwd->color || !fwd->depth || !fwd->normal || !fwd->opacity) return SOF_ERR_INVALID_ARG;
    if (!ws->fwd_valid || ws->fwd_n != scene->n || ws->fwd_views != n_views || !cams) return SOF_ERR_STATE;
    int tile, chunk, k, list_cap;
    if ((rc = resolve_opts(opts, &tile, &chunk, &k, &list_cap))) return rc;
    {
        // the workspace holds the sorted lists of its last forward only: the cameras and the output
        // images must be that forward's (two forwards on one workspace, then the first one's
        // backward, would replay the second's lists against the first's images)
        thread_local CamSet given;
        if ((rc = build_cams(cams, n_views, tile, opts->near_plane, &given))) return rc;
        if (memcmp(&given, &ws->fwd_cams, cams_bytes(n_views)) != 0) {
            snprintf(ws->err, sizeof(ws->err), "the cameras differ from the last forward's on this workspace");
            return SOF_ERR_STATE;
        }
        const sof_render_out &o = ws->fwd_out;
        if (fwd->color != o.color || fwd->depth != o.depth || fwd->normal != o.normal || fwd->opacity != o.opacity) {
            snprintf(ws->err, sizeof(ws->err), "the outputs are not those of the last forward on this workspace");
            return SOF_ERR_STATE;
        }
    }
    if (tile != ws->tile || chunk != ws->chunk || k != ws->k || list_cap != ws->list_cap ||
        ((opts->flags & SOF_FLAG_APPROX_ORDER) != 0) != ws->approx ||
        opts->near_plane != ws->near_plane ||
        opts->t_stop != ws->t_stop)
        return SOF_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ws->last_stream = s;
    const Layout &L = ws->L;
    const long long n = scene->n, n_rec = n * n_views;
    const int tiles = ws->cams.total_tiles;
    SceneDev sc{scene->means, scene->log_scales, scene->quats, scene->opacity_logits, scene->sh, n, scene->sh_degree};
    {
        SOF_PHASE(ws, SOF_PHASE_GRAD_REDUCE, s);
        SOF_CUDA(ws, launch_grad_copies_zero(L.grad_copies, L.total_dev + 4, ws->vis_cap, s));
    }
    CompositeParams p;
    memset(&p, 0, sizeof(p));
    p.cams = L.cams;
    p.records = L.records;
    p.pairs = L.pairs;
    p.ranges = L.ranges;
    p.prefix_end = L.prefix_end;
    p.prefix_key = L.prefix_key;
    p.tile_flag = L.tile_flag;
    p.near_plane = opts->near_plane;
    p.t_stop = opts->t_stop;
    for (int c = 0; c < 3; ++c) p.bg[c] = opts->bg[c];
    p.color = fwd->color;
    p.depth = fwd->depth;
    p.normal = fwd->normal;
    p.opacity = fwd->opacity;
    p.d_color = gin->d_color;
    p.d_depth = gin->d_depth;
    p.d_exact = gin->d_exact_depth;
    p.d_median = gin->d_median_depth;
    p.d_normal = gin->d_normal;
    p.d_opacity = gin->d_opacity;
    p.rgrad = L.grad_copies;
    p.vis_pos = L.vis_pos;
    p.vis_cap = (int)ws->vis_cap;
    p.status = L.status;
    p.ovf_mask = L.ovf_mask;
    p.ovf_list = L.ovf_list;
    p.ovf_count = L.total_dev + 3;
    p.ovf_list2 = L.ovf_list2;
    p.ovf_count2 = L.total_dev + 5;
    p.redo_count = L.redo;
    p.redo_tiles = L.redo + 1;
    p.hit_list = L.hit_list;
    p.list_cap = list_cap;
    p.pix_cnt = L.pix_cnt;
    p.approx = (opts->flags & SOF_FLAG_APPROX_ORDER) != 0;
    if (ws->losses && (gin->d_distortion || gin->d_extent)) {
        p.d_distortion = gin->d_distortion;
        p.d_extent = gin->d_extent;
        p.loss_sums = L.loss_sums;
    }
    {
        SOF_PHASE(ws, SOF_PHASE_REPLAY_BWD, s);
        SOF_CUDA(ws, launch_composite_replay(p, tiles, tile, s));
        if (gin->d_opacity_at_depth && fwd->opacity_at_depth && fwd->exact_depth) {
            p.exact_depth = fwd->exact_depth;
            p.opa = fwd->opacity_at_depth;
            p.d_opa = gin->d_opacity_at_depth;
            SOF_CUDA(ws, launch_opacity_at_depth(p, tiles, tile, true, s));
        }
    }
    {
        SOF_PHASE(ws, SOF_PHASE_COMPOSITE_BWD, s);
        SOF_CUDA(ws, launch_composite_bwd(p, tiles, tile, chunk, k, s));
        p.pass = 1;
        if (tile != 32) SOF_CUDA(ws, launch_composite_bwd(p, tiles, tile, chunk, kSecondPassK, s));
        SOF_CUDA(ws, launch_composite_fallback(p, tile, true, s));
    }
    {
        SOF_PHASE(ws, SOF_PHASE_GRAD_REDUCE, s);
        SOF_CUDA(ws, launch_grad_copies_reduce(L.grad_copies, L.total_dev + 4, ws->vis_cap, L.rgrad, s));
    }
    {
        SOF_PHASE(ws, SOF_PHASE_PREPROCESS_BWD, s);
        SOF_CUDA(ws, launch_preprocess_bwd(sc, L.cams, n_views, opts->near_plane, L.vflag, L.vis_pos,
                                           (int)ws->vis_cap, L.rgrad, *grad, s));
    }
    return SOF_OK;
}

namespace {

struct QLayout {
    size_t total = 0;
    CamSet *cams = nullptr;
    DevStatus *status = nullptr;
    // [2] Gaussian tile total, [4] records with tiles, [5] point tile total, [6] point blocks
    int *total_dev = nullptr;
    // 64-bit: [0] Gaussian binning items, [1] Gaussian pairs appended, [3] visible points appended
    unsigned long long *big = nullptr;
    float4 *records = nullptr;
    float4 *aux = nullptr;
    int4 *rects = nullptr;
    int *counts = nullptr;
    long long *offsets = nullptr;
    int *vflag = nullptr, *vis_pos = nullptr, *vis_list = nullptr, *vis_area = nullptr;
    void *scan_tmp = nullptr;
    unsigned *gtile = nullptr, *gkey = nullptr, *grec = nullptr;  // [pairs] unsorted Gaussian pairs (one block)
    unsigned *grank = nullptr;                                     // [pairs] their ranks in their tiles
    unsigned long long *gpairs = nullptr;                          // [pairs] z_min bits << 32 | record
    unsigned *ptile = nullptr, *pkey = nullptr, *pidx = nullptr;   // [points] unsorted visible points (one block)
    unsigned *prank = nullptr;                                     // [points] their ranks in their tiles
    unsigned long long *ppairs = nullptr;                          // [points] z bits << 32 | point
    int *gcounts = nullptr, *goffsets = nullptr, *gcursor = nullptr;  // [tiles]
    int *block_first = nullptr;  // [pairs / 256 + 1] the record of each binning CTA's first item
    int *pcounts = nullptr, *poffsets = nullptr, *pcursor = nullptr;  // [tiles]
    int2 *granges = nullptr, *pranges = nullptr;
    int *nb = nullptr, *bstart = nullptr;
    int2 *lut = nullptr;
};

long long max_point_blocks(long long n_points, int tiles) { return n_points / 256 + tiles + 1; }

// One view at a time: buffers sized for the largest view.
QLayout make_qlayout(char *base, long long n, long long pairs, long long n_points, int max_tiles) {
    QLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += al(bytes);
        return p;
    };
    auto ints = [&](long long k) { return reinterpret_cast<int *>(take((size_t)k * sizeof(int))); };
    auto u32 = [&](long long k) { return reinterpret_cast<unsigned *>(take((size_t)k * sizeof(unsigned))); };
    take(sizeof(Persist));  // the render's persistent state keeps its place
    L.cams = reinterpret_cast<CamSet *>(take(sizeof(CamSet)));
    L.status = reinterpret_cast<DevStatus *>(take(sizeof(DevStatus)));
    L.total_dev = ints(8);
    L.big = reinterpret_cast<unsigned long long *>(take(8 * sizeof(unsigned long long)));
    L.records = reinterpret_cast<float4 *>(take((size_t)n * kRecF4 * sizeof(float4)));
    L.aux = reinterpret_cast<float4 *>(take((size_t)n * sizeof(float4)));
    L.rects = reinterpret_cast<int4 *>(take((size_t)n * sizeof(int4)));
    L.counts = ints(n);
    L.offsets = reinterpret_cast<long long *>(take((size_t)n * sizeof(long long)));
    L.vflag = ints(n);
    L.vis_pos = ints(n);
    L.vis_list = ints(n);
    L.vis_area = ints(n);
    L.scan_tmp = take(scan_temp_bytes(std::max<long long>(n, max_tiles)));
    // the unsorted lists in one block: after the bucketing it serves the long-list sort as scratch
    L.gtile = u32(pairs * 4);
    L.gkey = L.gtile + pairs;
    L.grec = L.gkey + pairs;
    L.grank = L.grec + pairs;
    L.gpairs = reinterpret_cast<unsigned long long *>(take((size_t)pairs * 8));
    L.block_first = ints(pairs / 256 + 1);
    L.ptile = u32(n_points * 4);
    L.pkey = L.ptile + n_points;
    L.pidx = L.pkey + n_points;
    L.prank = L.pidx + n_points;
    L.ppairs = reinterpret_cast<unsigned long long *>(take((size_t)n_points * 8));
    L.gcounts = ints(max_tiles);
    L.goffsets = ints(max_tiles);
    L.gcursor = ints(max_tiles);
    L.pcounts = ints(max_tiles);
    L.poffsets = ints(max_tiles);
    L.pcursor = ints(max_tiles);
    L.granges = reinterpret_cast<int2 *>(take((size_t)max_tiles * sizeof(int2)));
    L.pranges = reinterpret_cast<int2 *>(take((size_t)max_tiles * sizeof(int2)));
    L.nb = ints(max_tiles);
    L.bstart = ints(max_tiles);
    L.lut = reinterpret_cast<int2 *>(take((size_t)max_point_blocks(n_points, max_tiles) * sizeof(int2)));
    L.total = off;
    return L;
}

int resolve_qopts(const sof_query_opts *o, int *tile) {
    *tile = o->tile == 0 ? 16 : o->tile;
    if (*tile != 8 && *tile != 16 && *tile != 32) return SOF_ERR_INVALID_ARG;
    if (o->flags & ~(SOF_QUERY_LEVEL_SET | SOF_QUERY_ASYNC | SOF_QUERY_PREPARED)) return SOF_ERR_INVALID_ARG;
    if (!(o->near_plane >= 0.f) || !(o->t_stop_query >= 0.f) || !(o->t_stop_query < 1.f)) return SOF_ERR_INVALID_ARG;
    return SOF_OK;
}

int max_view_tiles(const CamSet &cs) {
    int m = 1;
    for (int v = 0; v < cs.n_views; ++v) m = std::max(m, cs.cam[v].tiles_x * cs.cam[v].tiles_y);
    return m;
}

// Scratch of a prepared query (points only), laid out at `base` (after the resident region).
struct PQLayout {
    size_t total = 0;
    DevStatus *status = nullptr;
    int *total_dev = nullptr;  // [5] point tile total, [6] point blocks
    unsigned long long *big = nullptr;  // [3] visible points appended
    void *scan_tmp = nullptr;
    unsigned *ptile = nullptr, *pkey = nullptr, *pidx = nullptr, *prank = nullptr;
    unsigned long long *ppairs = nullptr;
    int *pcounts = nullptr, *poffsets = nullptr, *pcursor = nullptr;
    int2 *pranges = nullptr;
    int *nb = nullptr, *bstart = nullptr;
    int2 *lut = nullptr;
};

PQLayout make_pqlayout(char *base, long long n_points, int max_tiles) {
    PQLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += al(bytes);
        return p;
    };
    auto ints = [&](long long k) { return reinterpret_cast<int *>(take((size_t)k * sizeof(int))); };
    auto u32 = [&](long long k) { return reinterpret_cast<unsigned *>(take((size_t)k * sizeof(unsigned))); };
    L.status = reinterpret_cast<DevStatus *>(take(sizeof(DevStatus)));
    L.total_dev = ints(8);
    L.big = reinterpret_cast<unsigned long long *>(take(8 * sizeof(unsigned long long)));
    L.scan_tmp = take(scan_temp_bytes(max_tiles));
    L.ptile = u32(n_points * 4);
    L.pkey = L.ptile + n_points;
    L.pidx = L.pkey + n_points;
    L.prank = L.pidx + n_points;
    L.ppairs = reinterpret_cast<unsigned long long *>(take((size_t)n_points * 8));
    L.pcounts = ints(max_tiles);
    L.poffsets = ints(max_tiles);
    L.pcursor = ints(max_tiles);
    L.pranges = reinterpret_cast<int2 *>(take((size_t)max_tiles * sizeof(int2)));
    L.nb = ints(max_tiles);
    L.bstart = ints(max_tiles);
    L.lut = reinterpret_cast<int2 *>(take((size_t)max_point_blocks(n_points, max_tiles) * sizeof(int2)));
    L.total = off;
    return L;
}

// The buffers a level-set bisection of n_edges keeps at the end of the workspace (midpoints and
// their opacities).
size_t bisect_tail(long long n_edges) {
    return al((size_t)n_edges * 3 * sizeof(float)) + al((size_t)n_edges * sizeof(float)) + 256;
}

// The resident region of a prepared query: [persistent header][cameras][records of every view]
// [every view's sorted Gaussian pairs][every view's tile ranges]; returns its size.
size_t prep_region(long long n, int n_views, long long total_pairs, int max_tiles, size_t *cams_off, size_t *rec_off,
                   size_t *pair_off, size_t *range_off) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += al(bytes);
        return o;
    };
    take(sizeof(Persist));
    *cams_off = take(sizeof(CamSet));
    *rec_off = take((size_t)n_views * n * kRecF4 * sizeof(float4));
    *pair_off = take((size_t)total_pairs * 8);
    *range_off = take((size_t)n_views * max_tiles * sizeof(int2));
    return off;
}

long long fit_qpairs(size_t bytes, long long n, long long n_points, int tiles) {
    if (make_qlayout(nullptr, n, 0, n_points, tiles).total > bytes) return -1;
    long long lo = 0, hi = 1;
    while (make_qlayout(nullptr, n, hi, n_points, tiles).total <= bytes && hi < (1ll << 31)) hi *= 2;
    while (hi - lo > 1) {
        long long mid = (lo + hi) / 2;
        if (make_qlayout(nullptr, n, mid, n_points, tiles).total <= bytes) lo = mid;
        else hi = mid;
    }
    return std::min<long long>(lo, (1ll << 31) - 1);
}

}  // namespace

int sof_query_workspace_size(const sof_scene *scene, const sof_camera *cams, int n_views, int64_t n_points,
                             const sof_query_opts *opts, int64_t pair_capacity, size_t *bytes) {
    if (!bytes || !opts || pair_capacity < 0 || n_points < 0) return SOF_ERR_INVALID_ARG;
    int rc = validate_scene(scene, false);
    if (rc) return rc;
    int tile;
    if ((rc = resolve_qopts(opts, &tile))) return rc;
    thread_local CamSet tmp;
    if ((rc = build_cams(cams, n_views, tile, opts->near_plane, &tmp))) return rc;
    *bytes = make_qlayout(nullptr, scene->n, pair_capacity, n_points, max_view_tiles(tmp)).total;
    return SOF_OK;
}

int sof_query_prepare(const sof_scene *scene, const sof_camera *cams, int n_views, int64_t max_points,
                      const sof_query_opts *opts, sof_workspace *ws, void *stream) {
    if (!ws || !opts || max_points < 0 || max_points >= (1ll << 31)) return SOF_ERR_INVALID_ARG;
    ws->fwd_valid = false;
    ws->prep.valid = false;
    ws->required = 0;
    int rc = validate_scene(scene, false);
    if (rc) return rc;
    int tile;
    if ((rc = resolve_qopts(opts, &tile))) return rc;
    if ((rc = check_device(ws))) return rc;
    thread_local CamSet all;
    if ((rc = build_cams(cams, n_views, tile, opts->near_plane, &all))) return rc;
    const long long n = scene->n;
    if (n * (long long)n_views >= (1ll << 31)) return SOF_ERR_INVALID_ARG;  // record indices per view fit
    const int mt = max_view_tiles(all);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ws->last_stream = s;
    SceneDev sc{scene->means, scene->log_scales, scene->quats, scene->opacity_logits, nullptr, n, 0};
    auto single = [&](int v) {
        CamSet cs;
        cs.n_views = 1;
        cs.tile = tile;
        cs.cam[0] = all.cam[v];
        cs.cam[0].tile_base = 0;
        cs.cam[0].pix_base = 0;
        cs.total_tiles = cs.cam[0].tiles_x * cs.cam[0].tiles_y;
        return cs;
    };
    // sizing pass, at the front of the workspace: per view the binning items and the pairs that pass
    const size_t probe = make_qlayout(nullptr, n, 0, 0, mt).total;
    if (!ws->base || probe > ws->bytes) {
        ws->required = probe;
        return SOF_ERR_WORKSPACE_TOO_SMALL;
    }
    QLayout Ls = make_qlayout(ws->base, n, 0, 0, mt);
    ws->L = Layout();
    ws->L.status = Ls.status;
    SOF_CUDA(ws, cudaMemsetAsync(Ls.status, 0, sizeof(DevStatus), s));
    std::vector<long long> items(n_views), passing(n_views);
    thread_local CamSet cs;
    for (int v = 0; v < n_views; ++v) {
        cs = single(v);
        SOF_CUDA(ws, launch_set_cams(cs, Ls.cams, s));
        SOF_CUDA(ws, cudaMemsetAsync(Ls.total_dev, 0, 8 * sizeof(int), s));
        SOF_CUDA(ws, cudaMemsetAsync(Ls.big, 0, 8 * sizeof(unsigned long long), s));
        SOF_CUDA(ws, cudaMemsetAsync(Ls.vis_area, 0, (size_t)n * sizeof(int), s));
        SOF_CUDA(ws, launch_preprocess(sc, Ls.cams, cs, opts->near_plane, true, Ls.records, Ls.aux, Ls.rects,
                                       Ls.status, s));
        SOF_CUDA(ws, launch_rect_area(Ls.aux, Ls.rects, n, Ls.counts, Ls.vflag, s));
        SOF_CUDA(ws, launch_exclusive_scan(Ls.vflag, Ls.vis_pos, n, Ls.scan_tmp, Ls.total_dev + 4, s));
        SOF_CUDA(ws, launch_compact_visible(Ls.counts, Ls.vflag, Ls.vis_pos, n, Ls.vis_list, Ls.vis_area, n, nullptr,
                                            s));
        SOF_CUDA(ws, launch_exclusive_scan64(Ls.vis_area, Ls.offsets, n, Ls.scan_tmp,
                                             reinterpret_cast<long long *>(Ls.big), s));
        SOF_CUDA(ws, launch_bin_append(Ls.cams, n, Ls.records, Ls.aux, Ls.rects, Ls.vis_list, Ls.offsets,
                                       Ls.total_dev + 4, reinterpret_cast<const long long *>(Ls.big), 1ll << 62, true,
                                       opts->near_plane, 0, Ls.big + 2, nullptr, nullptr, nullptr, nullptr, nullptr,
                                       s, nullptr, nullptr));
        unsigned long long h[3] = {0, 0, 0};
        SOF_CUDA(ws, cudaMemcpyAsync(h, Ls.big, sizeof(h), cudaMemcpyDeviceToHost, s));
        SOF_CUDA(ws, cudaStreamSynchronize(s));
        items[v] = (long long)h[0];
        passing[v] = (long long)h[2];
        if (items[v] >= (1ll << 31) - 1024) {
            snprintf(ws->err, sizeof(ws->err), "view %d has %lld (Gaussian, tile) candidates: beyond 32-bit indexing",
                     v, items[v]);
            return SOF_ERR_INVALID_ARG;
        }
    }
    long long total_pairs = 0, max_items = 0;
    std::vector<long long> off(n_views + 1, 0);
    for (int v = 0; v < n_views; ++v) {
        off[v] = total_pairs;
        total_pairs += passing[v];
        max_items = std::max(max_items, items[v]);
    }
    off[n_views] = total_pairs;
    size_t cams_off, rec_off, pair_off, range_off;
    const size_t region = prep_region(n, n_views, total_pairs, mt, &cams_off, &rec_off, &pair_off, &range_off);
    // the build pass's scratch follows the resident region (its own records are not used); so does
    // the points' scratch of the prepared queries that follow
    const size_t need = region + std::max(make_qlayout(nullptr, n, max_items, 0, mt).total,
                                          make_pqlayout(nullptr, max_points, mt).total + bisect_tail(max_points));
    if (need > ws->bytes) {
        ws->required = need;
        return SOF_ERR_WORKSPACE_TOO_SMALL;
    }
    char *base = ws->base;
    QLayout Lb = make_qlayout(base + region, n, max_items, 0, mt);
    ws->L.status = Lb.status;
    SOF_CUDA(ws, cudaMemsetAsync(Lb.status, 0, sizeof(DevStatus), s));
    // the resident camera set: every view, each with its own tiles numbered from 0
    thread_local CamSet res;
    res = all;
    for (int v = 0; v < n_views; ++v) {
        res.cam[v].tile_base = 0;
        res.cam[v].pix_base = 0;
    }
    SOF_CUDA(ws, launch_set_cams(res, reinterpret_cast<CamSet *>(base + cams_off), s));
    for (int v = 0; v < n_views; ++v) {
        cs = single(v);
        const int tiles = cs.total_tiles;
        float4 *rec_v = reinterpret_cast<float4 *>(base + rec_off) + (size_t)v * n * kRecF4;
        unsigned long long *pairs_v = reinterpret_cast<unsigned long long *>(base + pair_off) + off[v];
        int2 *ranges_v = reinterpret_cast<int2 *>(base + range_off) + (size_t)v * mt;
        SOF_CUDA(ws, launch_set_cams(cs, Lb.cams, s));
        SOF_CUDA(ws, cudaMemsetAsync(Lb.total_dev, 0, 8 * sizeof(int), s));
        SOF_CUDA(ws, cudaMemsetAsync(Lb.big, 0, 8 * sizeof(unsigned long long), s));
        SOF_CUDA(ws, cudaMemsetAsync(Lb.gcounts, 0, (size_t)tiles * sizeof(int), s));
        SOF_CUDA(ws, cudaMemsetAsync(Lb.vis_area, 0, (size_t)n * sizeof(int), s));
        {
            SOF_PHASE(ws, SOF_PHASE_PREPROCESS, s);
            SOF_CUDA(ws, launch_preprocess(sc, Lb.cams, cs, opts->near_plane, true, rec_v, Lb.aux, Lb.rects,
                                           Lb.status, s));
        }
        {
            SOF_PHASE(ws, SOF_PHASE_SCAN, s);
            SOF_CUDA(ws, launch_rect_area(Lb.aux, Lb.rects, n, Lb.counts, Lb.vflag, s));
            SOF_CUDA(ws, launch_exclusive_scan(Lb.vflag, Lb.vis_pos, n, Lb.scan_tmp, Lb.total_dev + 4, s));
            SOF_CUDA(ws, launch_compact_visible(Lb.counts, Lb.vflag, Lb.vis_pos, n, Lb.vis_list, Lb.vis_area, n,
                                                nullptr, s));
            SOF_CUDA(ws, launch_exclusive_scan64(Lb.vis_area, Lb.offsets, n, Lb.scan_tmp,
                                                 reinterpret_cast<long long *>(Lb.big), s));
        }
        const long long *n_items_dev = reinterpret_cast<const long long *>(Lb.big);
        {
            SOF_PHASE(ws, SOF_PHASE_BIN_EMIT, s);
            SOF_CUDA(ws, launch_block_first(Lb.offsets, Lb.total_dev + 4, n_items_dev, n, items[v], Lb.block_first,
                                            s));
            SOF_CUDA(ws, launch_bin_append(Lb.cams, n, rec_v, Lb.aux, Lb.rects, Lb.vis_list, Lb.offsets,
                                           Lb.total_dev + 4, n_items_dev, items[v], true, opts->near_plane, max_items,
                                           Lb.big + 1, Lb.gtile, Lb.gkey, Lb.grec, Lb.gcounts, &Lb.status->n_dropped,
                                           s, Lb.block_first, nullptr, Lb.grank));
        }
        {
            SOF_PHASE(ws, SOF_PHASE_SORT, s);
            SOF_CUDA(ws, launch_exclusive_scan(Lb.gcounts, Lb.goffsets, tiles, Lb.scan_tmp, Lb.total_dev + 2, s));
            // the view's pairs land, sorted by (z_min, record) per tile, in its resident range
            SOF_CUDA(ws, launch_tile_buckets(Lb.gtile, Lb.gkey, Lb.grec, Lb.big + 1, std::max(passing[v], 1ll),
                                             Lb.gcounts, Lb.goffsets, tiles, ranges_v, Lb.gcursor, pairs_v,
                                             &Lb.status->n_pairs, s, nullptr, false,
                                             reinterpret_cast<unsigned long long *>(Lb.gtile), Lb.grank));
        }
    }
    {
        auto &P = ws->prep;
        P.valid = true;
        P.n = n;
        P.n_views = n_views;
        P.tile = tile;
        P.max_tiles = mt;
        P.near_plane = opts->near_plane;
        P.cams = all;
        P.pair_off = off;
        P.cams_dev = cams_off;
        P.records = rec_off;
        P.pairs = pair_off;
        P.ranges = range_off;
        P.end = region;
    }
    return SOF_OK;
}

}  // extern "C"

namespace {
// The query of points against the views sof_query_prepare left resident: per view, the points'
// projection, bucketing and block tables, then the integration against the view's resident sorted
// Gaussian lists. No host round trip (stream-ordered, capturable in a CUDA graph).
int prepared_query(const sof_scene *scene, const CamSet &all, const float *points, long long n_points,
                   const sof_query_opts *opts, int tile, float *opacity_out, int32_t *seen_count, sof_workspace *ws,
                   void *stream, size_t bytes) {
    const auto &P = ws->prep;
    if (!P.valid || P.n != scene->n || P.n_views != all.n_views || P.tile != tile || P.near_plane != opts->near_plane ||
        memcmp(&P.cams, &all, cams_bytes(all.n_views)) != 0) {
        snprintf(ws->err, sizeof(ws->err), "no matching sof_query_prepare on this workspace");
        return SOF_ERR_STATE;
    }
    const size_t need = P.end + make_pqlayout(nullptr, n_points, P.max_tiles).total;
    if (need > bytes) {
        ws->required = need + (ws->bytes - bytes);  // what the caller's own tail (if any) adds back
        return SOF_ERR_WORKSPACE_TOO_SMALL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ws->last_stream = s;
    char *base = ws->base;
    PQLayout L = make_pqlayout(base + P.end, n_points, P.max_tiles);
    ws->L = Layout();
    ws->L.status = L.status;
    const CamSet *cams_dev = reinterpret_cast<const CamSet *>(base + P.cams_dev);
    const float4 *records = reinterpret_cast<const float4 *>(base + P.records);
    const unsigned long long *pairs = reinterpret_cast<const unsigned long long *>(base + P.pairs);
    const int2 *ranges = reinterpret_cast<const int2 *>(base + P.ranges);
    SOF_CUDA(ws, cudaMemsetAsync(L.status, 0, sizeof(DevStatus), s));
    SOF_CUDA(ws, launch_fill(opacity_out, n_points, 1.0f, s));
    if (seen_count) SOF_CUDA(ws, cudaMemsetAsync(seen_count, 0, (size_t)n_points * sizeof(int32_t), s));
    for (int v = 0; v < all.n_views; ++v) {
        const int tiles = all.cam[v].tiles_x * all.cam[v].tiles_y;
        SOF_CUDA(ws, cudaMemsetAsync(L.total_dev, 0, 8 * sizeof(int), s));
        SOF_CUDA(ws, cudaMemsetAsync(L.big, 0, 8 * sizeof(unsigned long long), s));
        SOF_CUDA(ws, cudaMemsetAsync(L.pcounts, 0, (size_t)tiles * sizeof(int), s));
        {
            SOF_PHASE(ws, SOF_PHASE_QUERY_POINTS, s);
            SOF_CUDA(ws, launch_point_append(cams_dev, v, points, n_points, opts->near_plane, seen_count, L.big + 3,
                                             L.ptile, L.pkey, L.pidx, L.prank, L.pcounts, s));
            SOF_CUDA(ws, launch_exclusive_scan(L.pcounts, L.poffsets, tiles, L.scan_tmp, L.total_dev + 5, s));
            SOF_CUDA(ws, launch_tile_buckets(L.ptile, L.pkey, L.pidx, L.big + 3, n_points, L.pcounts, L.poffsets,
                                             tiles, L.pranges, L.pcursor, L.ppairs, nullptr, s, nullptr, true,
                                             reinterpret_cast<unsigned long long *>(L.ptile), L.prank));
            SOF_CUDA(ws, launch_tile_blocks(L.pcounts, tiles, L.nb, s));
            SOF_CUDA(ws, launch_exclusive_scan(L.nb, L.bstart, tiles, L.scan_tmp, L.total_dev + 6, s));
            SOF_CUDA(ws, launch_fill_lut(L.nb, L.bstart, tiles, L.lut, s));
        }
        SOF_PHASE(ws, SOF_PHASE_QUERY_INTEGRATE, s);
        SOF_CUDA(ws, launch_integrate(cams_dev, v, records + (size_t)v * P.n * kRecF4, pairs + P.pair_off[v],
                                      ranges + (size_t)v * P.max_tiles, L.ppairs, L.pranges, L.lut, L.total_dev + 6,
                                      max_point_blocks(n_points, tiles), points, opts->near_plane, opts->t_stop_query,
                                      (opts->flags & SOF_QUERY_LEVEL_SET) != 0, opacity_out, L.status,
                                      n_points / std::max(tiles, 1), s));
    }
    return SOF_OK;
}

// The query over the first `bytes` of the workspace (the level-set bisection keeps its own buffers
// after them).
int query_impl(const sof_scene *scene, const sof_camera *cams, int n_views, const float *points, int64_t n_points,
               const sof_query_opts *opts, float *opacity_out, int32_t *seen_count, sof_workspace *ws, void *stream,
               size_t bytes) {
    if (!ws || !opts || n_points < 0 || (n_points > 0 && (!points || !opacity_out))) return SOF_ERR_INVALID_ARG;
    if (n_points >= (1ll << 31)) return SOF_ERR_INVALID_ARG;
    ws->fwd_valid = false;
    ws->required = 0;
    int rc = validate_scene(scene, false);
    if (rc) return rc;
    int tile;
    if ((rc = resolve_qopts(opts, &tile))) return rc;
    if ((rc = check_device(ws))) return rc;
    thread_local CamSet all;
    if ((rc = build_cams(cams, n_views, tile, opts->near_plane, &all))) return rc;
    if (opts->flags & SOF_QUERY_PREPARED)
        return prepared_query(scene, all, points, n_points, opts, tile, opacity_out, seen_count, ws, stream, bytes);
    ws->prep.valid = false;  // this query lays out its scratch from the front of the workspace
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ws->last_stream = s;
    const long long n = scene->n;
    const int mt = max_view_tiles(all);
    long long cap = fit_qpairs(bytes, n, n_points, mt);
    if (cap < 0 || !ws->base) {
        ws->required = make_qlayout(nullptr, n, std::max<long long>(n * 4, 1024), n_points, mt).total;
        return SOF_ERR_WORKSPACE_TOO_SMALL;
    }
    QLayout L = make_qlayout(ws->base, n, cap, n_points, mt);
    const bool async = (opts->flags & SOF_QUERY_ASYNC) != 0;
    ws->L = Layout();
    ws->L.status = L.status;
    SceneDev sc{scene->means, scene->log_scales, scene->quats, scene->opacity_logits, nullptr, n, 0};
    SOF_CUDA(ws, cudaMemsetAsync(L.status, 0, sizeof(DevStatus), s));
    SOF_CUDA(ws, launch_fill(opacity_out, n_points, 1.0f, s));
    if (seen_count) SOF_CUDA(ws, cudaMemsetAsync(seen_count, 0, (size_t)n_points * sizeof(int32_t), s));
    for (int v = 0; v < n_views; ++v) {
        // this view alone, tiles numbered from 0
        CamSet &cs = ws->cams;
        cs.n_views = 1;
        cs.tile = tile;
        cs.cam[0] = all.cam[v];
        cs.cam[0].tile_base = 0;
        cs.cam[0].pix_base = 0;
        const int tiles = cs.cam[0].tiles_x * cs.cam[0].tiles_y;
        cs.total_tiles = tiles;
        SOF_CUDA(ws, launch_set_cams(cs, L.cams, s));
        SOF_CUDA(ws, cudaMemsetAsync(L.total_dev, 0, 8 * sizeof(int), s));
        SOF_CUDA(ws, cudaMemsetAsync(L.big, 0, 8 * sizeof(unsigned long long), s));
        SOF_CUDA(ws, cudaMemsetAsync(L.gcounts, 0, (size_t)tiles * sizeof(int), s));
        SOF_CUDA(ws, cudaMemsetAsync(L.pcounts, 0, (size_t)tiles * sizeof(int), s));
        SOF_CUDA(ws, cudaMemsetAsync(L.vis_area, 0, (size_t)n * sizeof(int), s));
        {
            SOF_PHASE(ws, SOF_PHASE_PREPROCESS, s);
            SOF_CUDA(ws, launch_preprocess(sc, L.cams, cs, opts->near_plane, true, L.records, L.aux, L.rects,
                                           L.status, s));
        }
        {
            SOF_PHASE(ws, SOF_PHASE_BIN_COUNT, s);
            SOF_CUDA(ws, launch_rect_area(L.aux, L.rects, n, L.counts, L.vflag, s));
        }
        {
            SOF_PHASE(ws, SOF_PHASE_SCAN, s);
            SOF_CUDA(ws, launch_exclusive_scan(L.vflag, L.vis_pos, n, L.scan_tmp, L.total_dev + 4, s));
            SOF_CUDA(ws, launch_compact_visible(L.counts, L.vflag, L.vis_pos, n, L.vis_list, L.vis_area, n,
                                                nullptr, s));
            SOF_CUDA(ws, launch_exclusive_scan64(L.vis_area, L.offsets, n, L.scan_tmp,
                                                 reinterpret_cast<long long *>(L.big), s));
        }
        {
            // points do not depend on the Gaussians: queued before the view's one host round trip
            SOF_PHASE(ws, SOF_PHASE_QUERY_POINTS, s);
            SOF_CUDA(ws, launch_point_append(L.cams, 0, points, n_points, opts->near_plane, seen_count,
                                             L.big + 3, L.ptile, L.pkey, L.pidx, L.prank, L.pcounts, s));
            SOF_CUDA(ws, launch_exclusive_scan(L.pcounts, L.poffsets, tiles, L.scan_tmp, L.total_dev + 5, s));
            // points in (tile, z) order only to group similar depths in a CTA: each point is
            // integrated on its own, so long tiles are sorted in blocks, not merged
            SOF_CUDA(ws, launch_tile_buckets(L.ptile, L.pkey, L.pidx, L.big + 3, n_points, L.pcounts,
                                             L.poffsets, tiles, L.pranges, L.pcursor, L.ppairs, nullptr, s, nullptr,
                                             true, reinterpret_cast<unsigned long long *>(L.ptile), L.prank));
            SOF_CUDA(ws, launch_tile_blocks(L.pcounts, tiles, L.nb, s));
            SOF_CUDA(ws, launch_exclusive_scan(L.nb, L.bstart, tiles, L.scan_tmp, L.total_dev + 6, s));
            SOF_CUDA(ws, launch_fill_lut(L.nb, L.bstart, tiles, L.lut, s));
        }
        long long bound = cap;  // without the round trip: as many items as the capacity holds pairs
        if (!async) {
            // the view's one host round trip: the pair bound decides whether the workspace suffices
            long long hb = 0;
            SOF_CUDA(ws, cudaMemcpyAsync(&hb, L.big, sizeof(hb), cudaMemcpyDeviceToHost, s));
            SOF_CUDA(ws, cudaStreamSynchronize(s));
            if (hb < 0) return SOF_ERR_INVALID_ARG;
            if (hb > cap) {
                ws->required = make_qlayout(nullptr, n, (long long)hb + hb / 8 + 1024, n_points, mt).total;
                return SOF_ERR_WORKSPACE_TOO_SMALL;
            }
            // a view without pairs still runs the integration: the points it sees have opacity 0
            // there, which lowers their minimum over the views
            bound = hb;
        }
        {
            SOF_PHASE(ws, SOF_PHASE_BIN_EMIT, s);
            const long long *n_items_dev = reinterpret_cast<const long long *>(L.big);
            SOF_CUDA(ws, launch_block_first(L.offsets, L.total_dev + 4, n_items_dev, n, bound, L.block_first, s));
            SOF_CUDA(ws, launch_bin_append(L.cams, n, L.records, L.aux, L.rects, L.vis_list, L.offsets,
                                           L.total_dev + 4, n_items_dev, bound, true, opts->near_plane, cap,
                                           L.big + 1, L.gtile, L.gkey, L.grec, L.gcounts,
                                           async ? &L.status->n_dropped : nullptr, s, L.block_first, L.pcounts,
                                           L.grank));
        }
        {
            SOF_PHASE(ws, SOF_PHASE_SORT, s);
            SOF_CUDA(ws, launch_exclusive_scan(L.gcounts, L.goffsets, tiles, L.scan_tmp, L.total_dev + 2, s));
            SOF_CUDA(ws, launch_tile_buckets(L.gtile, L.gkey, L.grec, L.big + 1, bound, L.gcounts,
                                             L.goffsets, tiles, L.granges, L.gcursor, L.gpairs,
                                             &L.status->n_pairs, s, nullptr, false,
                                             reinterpret_cast<unsigned long long *>(L.gtile), L.grank));
        }
        SOF_PHASE(ws, SOF_PHASE_QUERY_INTEGRATE, s);
        SOF_CUDA(ws, launch_integrate(L.cams, 0, L.records, L.gpairs, L.granges, L.ppairs, L.pranges, L.lut,
                                      L.total_dev + 6, max_point_blocks(n_points, tiles), points, opts->near_plane,
                                      opts->t_stop_query, (opts->flags & SOF_QUERY_LEVEL_SET) != 0, opacity_out,
                                      L.status, n_points / std::max(tiles, 1), s));
    }
    return SOF_OK;
}
}  // namespace

extern "C" {

int sof_opacity_query(const sof_scene *scene, const sof_camera *cams, int n_views, const float *points,
                      int64_t n_points, const sof_query_opts *opts, float *opacity_out, int32_t *seen_count,
                      sof_workspace *ws, void *stream) {
    if (!ws) return SOF_ERR_INVALID_ARG;
    return query_impl(scene, cams, n_views, points, n_points, opts, opacity_out, seen_count, ws, stream, ws->bytes);
}

int sof_level_set_bisect(const sof_scene *scene, const sof_camera *cams, int n_views, float *inside, float *outside,
                         int64_t n_edges, int iterations, const sof_query_opts *opts, sof_workspace *ws, void *stream) {
    if (!ws || !opts || n_edges < 0 || iterations < 0 || iterations > 64) return SOF_ERR_INVALID_ARG;
    if (n_edges > 0 && (!inside || !outside)) return SOF_ERR_INVALID_ARG;
    if (!(opts->flags & SOF_QUERY_LEVEL_SET)) return SOF_ERR_INVALID_ARG;
    if (n_edges >= (1ll << 31)) return SOF_ERR_INVALID_ARG;
    ws->required = 0;
    // the midpoints [n_edges][3] and their opacities [n_edges] sit at the end of the workspace
    const size_t tail = bisect_tail(n_edges);
    const size_t qbytes = ws->bytes > tail ? ((ws->bytes - tail) & ~(size_t)255) : 0;
    if (n_edges == 0 || iterations == 0) return SOF_OK;
    if (!ws->base || qbytes == 0) {
        // no room for the query beside the edge buffers: a query over no bytes only reports its need
        const int rc = query_impl(scene, cams, n_views, inside, n_edges, opts, inside, nullptr, ws, stream, 0);
        if (rc == SOF_ERR_WORKSPACE_TOO_SMALL) ws->required += tail + 256;
        return rc ? rc : SOF_ERR_WORKSPACE_TOO_SMALL;
    }
    float *mid = reinterpret_cast<float *>(ws->base + qbytes);
    float *o_mid = reinterpret_cast<float *>(reinterpret_cast<char *>(mid) + al((size_t)n_edges * 3 * sizeof(float)));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int it = 0; it < iterations; ++it) {
        SOF_CUDA(ws, launch_midpoints(inside, outside, n_edges, mid, s));
        const int rc = query_impl(scene, cams, n_views, mid, n_edges, opts, o_mid, nullptr, ws, stream, qbytes);
        if (rc == SOF_ERR_WORKSPACE_TOO_SMALL) {
            ws->required += tail + 256;
            return rc;
        }
        if (rc) return rc;
        SOF_CUDA(ws, launch_bisect_update(inside, outside, mid, o_mid, n_edges, s));
    }
    return SOF_OK;
}

}  // extern "C"

// ------------------------------------------------------------- forward render without allocation
// Some callers cannot allocate device memory at all: code running where the CUDA allocator is
// off limits (a host that pre-reserves all device memory for itself, a plugin inside a runtime that
// forbids cudaMalloc/cudaFree, or a memory budget fixed at start-up). sof_render_fwd_noalloc lets
// them render small scenes anyway: its scratch is a fixed device array compiled into this library,
// so the call itself never allocates. The array lives on every GPU that loads the library until the
// process exits, and all calls on a device share it.
static __device__ __align__(256) unsigned char g_sof_noalloc_scratch[SOF_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNoallocDevices = 16;
struct NoallocSlot {
    std::mutex m;
    bool ready = false;
    sof_workspace ws;  // host-side handle bound to this device's copy of the array
};
NoallocSlot g_noalloc[kNoallocDevices];
// the message of the last failed no-allocation call on any device (the calls have no handle to
// read it from); written under the failing device's lock
thread_local char g_noalloc_err[512] = {0};
void noalloc_note_error(const char *msg) { snprintf(g_noalloc_err, sizeof(g_noalloc_err), "%s", msg); }
}  // namespace

extern "C" int sof_render_fwd_noalloc(const sof_scene *scene, const sof_camera *cams, int n_views,
                                      const sof_render_opts *opts, const sof_render_out *out,
                                      size_t *required_bytes, void *stream) {
    if (required_bytes) *required_bytes = 0;
    int rc = check_device(nullptr);
    if (rc != SOF_OK) return rc;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocDevices) {
        cudaGetLastError();
        return SOF_ERR_NO_DEVICE;
    }
    NoallocSlot &slot = g_noalloc[dev];
    std::lock_guard<std::mutex> lock(slot.m);
    slot.ws.err[0] = 0;
    if (!slot.ready) {
        // once per device, with that device current: the device address of the array (in host
        // code the array's name is only a host-side stand-in and must not be passed to a kernel)
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_sof_noalloc_scratch);
        if (e != cudaSuccess) {
            rc = cuda_fail(&slot.ws, e, "cudaGetSymbolAddress(g_sof_noalloc_scratch)");
            noalloc_note_error(slot.ws.err);
            return rc;
        }
        rc = sof_workspace_bind(&slot.ws, ptr, SOF_NOALLOC_SCRATCH_BYTES);
        if (rc != SOF_OK) return rc;
        slot.ready = true;
    }
    // Every call is sized on its own (whether a scene fits does not depend on earlier calls) and
    // checked: the pair bound is read back, so a scene that does not fit is refused with
    // SOF_ERR_WORKSPACE_TOO_SMALL instead of being rendered with pairs dropped. The array keeps no
    // gradient copies or replay lists: no backward can follow this forward.
    slot.ws.vis_hint = 0;
    if (!opts) return SOF_ERR_INVALID_ARG;
    sof_render_opts o = *opts;
    o.flags |= SOF_FLAG_CHECKED;
    o.replay_cap = -1;
    // The forward path clears everything it needs zeroed (counters, tile ranges) on every call.
    rc = render_fwd_impl(scene, cams, n_views, &o, out, &slot.ws, stream, kFwdChecked, false, nullptr);
    if (rc == SOF_ERR_WORKSPACE_TOO_SMALL && required_bytes) *required_bytes = slot.ws.required;
    if (rc < 0) noalloc_note_error(slot.ws.err[0] ? slot.ws.err : sof_error_string(rc));
    return rc;
}

extern "C" const char *sof_noalloc_last_error(void) { return g_noalloc_err; }
