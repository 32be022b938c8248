// Host drivers of the batched training step (include/sof.h): the step of many views captured in a
// CUDA graph (sof_graph_*) and the autotuner of the composite's (tile, chunk, reorder_k)
// (sof_autotune). Both only order calls of the render entry points; no data is touched here.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sof_internal.cuh"

using namespace sof;

struct sof_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

long long view_pixels(const sof_camera &c) { return (long long)c.width * c.height; }

// The groups of views one step renders: [first, first + count) with its packed pixel offset.
struct Group {
    int first, count;
    long long pix;
};

std::vector<Group> make_groups(const sof_camera *cams, int n_views, int views_per_call) {
    std::vector<Group> g;
    const int vpc = views_per_call <= 0 ? n_views : views_per_call;
    long long pix = 0;
    for (int v = 0; v < n_views; v += vpc) {
        const int k = std::min(vpc, n_views - v);
        g.push_back({v, k, pix});
        for (int i = 0; i < k; ++i) pix += view_pixels(cams[v + i]);
    }
    return g;
}

float *at(float *p, long long off) { return p ? p + off : nullptr; }
const float *at(const float *p, long long off) { return p ? p + off : nullptr; }
int32_t *at(int32_t *p, long long off) { return p ? p + off : nullptr; }

// The slices of the packed outputs and upstream gradients that group g writes and reads.
void slice(const sof_render_out &out, const sof_render_grad_in &gin, long long pix, sof_render_out *o,
           sof_render_grad_in *gi) {
    *o = out;
    o->color = at(out.color, 3 * pix);
    o->normal = at(out.normal, 3 * pix);
    o->depth = at(out.depth, pix);
    o->exact_depth = at(out.exact_depth, pix);
    o->median_depth = at(out.median_depth, pix);
    o->opacity = at(out.opacity, pix);
    o->n_contrib = at(out.n_contrib, pix);
    o->distortion = at(out.distortion, pix);
    o->extent = at(out.extent, pix);
    o->opacity_at_depth = at(out.opacity_at_depth, pix);
    *gi = gin;
    gi->d_color = at(gin.d_color, 3 * pix);
    gi->d_normal = at(gin.d_normal, 3 * pix);
    gi->d_depth = at(gin.d_depth, pix);
    gi->d_exact_depth = at(gin.d_exact_depth, pix);
    gi->d_median_depth = at(gin.d_median_depth, pix);
    gi->d_opacity = at(gin.d_opacity, pix);
    gi->d_distortion = at(gin.d_distortion, pix);
    gi->d_extent = at(gin.d_extent, pix);
    gi->d_opacity_at_depth = at(gin.d_opacity_at_depth, pix);
}

struct Step {
    const sof_scene *scene;
    const sof_camera *cams;
    int n_views;
    std::vector<Group> groups;
    sof_render_opts opts;  // stream-ordered (SOF_FLAG_CHECKED cleared)
    sof_render_out out;
    sof_render_grad_in gin;
    sof_scene_grad grad;
    bool zero_grads;
    sof_workspace *ws;
};

// Sizes the workspace for every group: SOF_OK if the bound workspace holds the largest group's
// step, else SOF_ERR_WORKSPACE_TOO_SMALL with the size recorded (or the first error). Two rounds:
// the capacity hints a reservation leaves only grow, and every group's size is taken with the
// hints of all groups (the groups share the workspace and its hints).
int reserve_all(const Step &st, cudaStream_t s) {
    size_t need = 0;
    for (int round = 0; round < 2; ++round) {
        need = 0;
        for (const Group &g : st.groups) {
            size_t b = 0;
            const int rc = sof_workspace_reserve(st.ws, st.scene, st.cams + g.first, g.count, &st.opts, s, &b);
            if (rc != SOF_OK) return rc;
            need = std::max(need, b);
        }
        if (st.groups.size() < 2) break;
    }
    if (need > workspace_bytes(st.ws)) {
        workspace_set_required(st.ws, need);
        return SOF_ERR_WORKSPACE_TOO_SMALL;
    }
    return SOF_OK;
}

// One step queued on s: zeroing, clearing the dropped counter, per group forward then backward.
int queue_step(const Step &st, cudaStream_t s) {
    int rc = sof_workspace_clear_dropped(st.ws, s);
    if (rc != SOF_OK) return rc;
    if (st.zero_grads) {
        const long long n = st.scene->n;
        const long long k = (long long)(st.scene->sh_degree + 1) * (st.scene->sh_degree + 1);
        struct {
            float *p;
            long long count;
        } z[5] = {{st.grad.d_means, 3 * n}, {st.grad.d_log_scales, 3 * n}, {st.grad.d_quats, 4 * n},
                  {st.grad.d_opacity_logits, n}, {st.grad.d_sh, 3 * k * n}};
        for (auto &b : z)
            if (b.p && b.count > 0 && cudaMemsetAsync(b.p, 0, (size_t)b.count * sizeof(float), s) != cudaSuccess)
                return SOF_ERR_CUDA;
    }
    for (const Group &g : st.groups) {
        sof_render_out o;
        sof_render_grad_in gi;
        slice(st.out, st.gin, g.pix, &o, &gi);
        rc = sof_render_fwd(st.scene, st.cams + g.first, g.count, &st.opts, &o, st.ws, s);
        if (rc < 0) return rc;
        rc = sof_render_bwd(st.scene, st.cams + g.first, g.count, &st.opts, &o, &gi, &st.grad, st.ws, s);
        if (rc < 0) return rc;
    }
    return SOF_OK;
}

int make_step(const sof_scene *scene, const sof_camera *cams, int n_views, int views_per_call,
              const sof_render_opts *opts, const sof_render_out *out, const sof_render_grad_in *grad_in,
              const sof_scene_grad *grad, int zero_grads, sof_workspace *ws, Step *st) {
    if (!scene || !cams || !opts || !out || !grad_in || !grad || !ws || n_views < 1 || n_views > SOF_MAX_VIEWS ||
        views_per_call < 0)
        return SOF_ERR_INVALID_ARG;
    st->scene = scene;
    st->cams = cams;
    st->n_views = n_views;
    st->groups = make_groups(cams, n_views, views_per_call);
    st->opts = *opts;
    st->opts.flags &= ~SOF_FLAG_CHECKED;
    st->out = *out;
    st->gin = *grad_in;
    st->grad = *grad;
    st->zero_grads = zero_grads != 0;
    st->ws = ws;
    return SOF_OK;
}

// Candidates of the autotuner: the (tile, chunk, reorder_k) triples the composite is instantiated for.
constexpr int kCand[SOF_AUTOTUNE_CANDIDATES][3] = {{16, 64, 16}, {16, 32, 16}, {16, 128, 16}, {16, 64, 8},
                                                   {16, 64, 32}, {16, 32, 8},  {16, 32, 32}, {8, 64, 16},
                                                   {8, 64, 32},  {32, 64, 8},  {32, 64, 16}};

std::string signature(const sof_scene *scene, const sof_camera *cams, int n_views, int views_per_call,
                      const sof_render_opts *b) {
    char buf[256];
    snprintf(buf, sizeof(buf), "n=%lld;sh=%d;vpc=%d;near=%g;stop=%g;flags=%u;cap=%d;prefix=%d;views=",
             (long long)scene->n, scene->sh_degree, views_per_call, b->near_plane, b->t_stop,
             b->flags & ~SOF_FLAG_CHECKED, b->replay_cap, b->sort_prefix);
    std::string s = buf;
    for (int v = 0; v < n_views; ++v) {
        snprintf(buf, sizeof(buf), "%s%dx%d", v ? "," : "", cams[v].width, cams[v].height);
        s += buf;
    }
    return s;
}

// The last cached line of this signature: "signature tile chunk reorder_k ms".
bool cache_lookup(const char *path, const std::string &sig, int *t, int *c, int *k, float *ms) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    bool found = false;
    std::vector<char> line(1 << 16);
    while (fgets(line.data(), (int)line.size(), f)) {
        const char *sp = strchr(line.data(), ' ');
        if (!sp || (size_t)(sp - line.data()) != sig.size() || strncmp(line.data(), sig.c_str(), sig.size()) != 0)
            continue;
        int a, b, d;
        float m;
        if (sscanf(sp + 1, "%d %d %d %f", &a, &b, &d, &m) == 4) {
            *t = a;
            *c = b;
            *k = d;
            *ms = m;
            found = true;
        }
    }
    fclose(f);
    return found;
}

}  // namespace

extern "C" {

int sof_graph_capture(const sof_scene *scene, const sof_camera *cams, int n_views, int views_per_call,
                      const sof_render_opts *opts, const sof_render_out *out, const sof_render_grad_in *grad_in,
                      const sof_scene_grad *grad, int zero_grads, sof_workspace *ws, void *stream,
                      sof_graph **graph) {
    if (!graph || !stream) return SOF_ERR_INVALID_ARG;
    *graph = nullptr;
    Step st;
    int rc = make_step(scene, cams, n_views, views_per_call, opts, out, grad_in, grad, zero_grads, ws, &st);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((rc = reserve_all(st, s))) return rc;
    // eager run: configures every kernel's attributes before the capture
    if ((rc = queue_step(st, s))) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SOF_ERR_CUDA;
    const bool timing = workspace_timing(ws);
    sof_workspace_set_timing(ws, 0);
    sof_graph *g = new sof_graph();
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        sof_workspace_set_timing(ws, timing);
        delete g;
        workspace_note(ws, cudaGetErrorString(e));
        return SOF_ERR_CUDA;
    }
    rc = queue_step(st, s);
    e = cudaStreamEndCapture(s, &g->graph);  // always ends the capture, also after an error
    sof_workspace_set_timing(ws, timing);
    if (rc == SOF_OK && e != cudaSuccess) rc = SOF_ERR_CUDA;
    if (rc == SOF_OK && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) rc = SOF_ERR_CUDA;
    if (rc != SOF_OK) {
        cudaGetLastError();
        sof_graph_destroy(g);
        return rc;
    }
    *graph = g;
    return SOF_OK;
}

int sof_graph_launch(sof_graph *graph, void *stream) {
    if (!graph || !graph->exec) return SOF_ERR_INVALID_ARG;
    return cudaGraphLaunch(graph->exec, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? SOF_OK
                                                                                                : SOF_ERR_CUDA;
}

int sof_graph_destroy(sof_graph *graph) {
    if (!graph) return SOF_OK;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
    return SOF_OK;
}

int sof_autotune_candidate(int index, int *tile, int *chunk, int *reorder_k) {
    if (index < 0 || index >= SOF_AUTOTUNE_CANDIDATES || !tile || !chunk || !reorder_k) return SOF_ERR_INVALID_ARG;
    *tile = kCand[index][0];
    *chunk = kCand[index][1];
    *reorder_k = kCand[index][2];
    return SOF_OK;
}

int sof_autotune(const sof_scene *scene, const sof_camera *cams, int n_views, int views_per_call,
                 const sof_render_opts *base, const sof_render_out *out, const sof_render_grad_in *grad_in,
                 const sof_scene_grad *grad, int reps, const char *cache_path, sof_workspace *ws, void *stream,
                 sof_render_opts *best, float *ms) {
    if (!best || reps < 1) return SOF_ERR_INVALID_ARG;
    Step st;
    int rc = make_step(scene, cams, n_views, views_per_call, base, out, grad_in, grad, 1, ws, &st);
    if (rc) return rc;
    for (int i = 0; i < SOF_AUTOTUNE_CANDIDATES; ++i)
        if (ms) ms[i] = -1.f;
    const std::string sig = signature(scene, cams, n_views, views_per_call, base);
    int ct, cc, ck;
    float cms;
    if (cache_path && cache_lookup(cache_path, sig, &ct, &cc, &ck, &cms)) {
        *best = *base;
        best->tile = ct;
        best->chunk = cc;
        best->reorder_k = ck;
        for (int i = 0; i < SOF_AUTOTUNE_CANDIDATES; ++i)
            if (ms && kCand[i][0] == ct && kCand[i][1] == cc && kCand[i][2] == ck) ms[i] = cms;
        return SOF_OK;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // size for every usable triple before timing any
    bool usable[SOF_AUTOTUNE_CANDIDATES];
    size_t need = 0;
    for (int round = 0; round < 2; ++round) {  // the second with the hints of every candidate
        need = 0;
        for (int i = 0; i < SOF_AUTOTUNE_CANDIDATES; ++i) {
            Step c = st;
            c.opts.tile = kCand[i][0];
            c.opts.chunk = kCand[i][1];
            c.opts.reorder_k = kCand[i][2];
            usable[i] = false;
            for (const Group &g : c.groups) {
                size_t b = 0;
                rc = sof_workspace_reserve(ws, scene, cams + g.first, g.count, &c.opts, s, &b);
                if (rc == SOF_ERR_INVALID_ARG) break;  // refused for this workload
                if (rc != SOF_OK) return rc;
                need = std::max(need, b);
            }
            usable[i] = rc == SOF_OK;
        }
    }
    if (need > workspace_bytes(ws)) {
        workspace_set_required(ws, need);
        return SOF_ERR_WORKSPACE_TOO_SMALL;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return SOF_ERR_CUDA;
    }
    int best_i = -1;
    float best_ms = 0.f;
    rc = SOF_OK;
    for (int i = 0; i < SOF_AUTOTUNE_CANDIDATES && rc == SOF_OK; ++i) {
        if (!usable[i]) continue;
        Step c = st;
        c.opts.tile = kCand[i][0];
        c.opts.chunk = kCand[i][1];
        c.opts.reorder_k = kCand[i][2];
        if ((rc = queue_step(c, s))) break;  // warm-up
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = SOF_ERR_CUDA;
        for (int r = 0; r < reps && rc == SOF_OK; ++r) rc = queue_step(c, s);
        if (rc != SOF_OK) break;
        float el = 0.f;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&el, e0, e1) != cudaSuccess) {
            rc = SOF_ERR_CUDA;
            break;
        }
        const float per = el / reps;
        if (ms) ms[i] = per;
        if (best_i < 0 || per < best_ms) {
            best_i = i;
            best_ms = per;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SOF_OK) return rc;
    if (best_i < 0) {
        workspace_note(ws, "no instantiated (tile, chunk, reorder_k) renders this workload");
        return SOF_ERR_INVALID_ARG;
    }
    *best = *base;
    best->tile = kCand[best_i][0];
    best->chunk = kCand[best_i][1];
    best->reorder_k = kCand[best_i][2];
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s %d %d %d %.6g\n", sig.c_str(), best->tile, best->chunk, best->reorder_k, best_ms);
            fclose(f);
        }
    }
    return SOF_OK;
}

}  // extern "C"
