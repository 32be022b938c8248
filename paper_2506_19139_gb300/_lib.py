"""ctypes binding of the C-ABI in include/sof.h: the same names, argument marshalling only.

Loads the in-tree libsof.so built by paper_2506_19139_gb300.build. There is no fallback: if the
library or a CUDA device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsof.so")

SOF_OK = 0
SOF_WARN_INEXACT = 1
SOF_ERR_INVALID_ARG = -1
SOF_ERR_CUDA = -2
SOF_ERR_WORKSPACE_TOO_SMALL = -3
SOF_ERR_NOT_IMPLEMENTED = -4
SOF_ERR_NO_DEVICE = -5
SOF_ERR_STATE = -6
SOF_MAX_VIEWS = 128
SOF_FLAG_MEDIAN_DEPTH = 1
SOF_FLAG_ASYNC = 2
SOF_FLAG_APPROX_ORDER = 4
SOF_FLAG_CHECKED = 8
SOF_AUTOTUNE_CANDIDATES = 11
SOF_QUERY_LEVEL_SET = 1
SOF_QUERY_ASYNC = 2
SOF_QUERY_PREPARED = 4


class sof_scene(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64), ("sh_degree", C.c_int32)]


class sof_camera(C.Structure):
    _fields_ = [("world_to_cam", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class sof_render_opts(C.Structure):
    _fields_ = [("near_plane", C.c_float), ("t_stop", C.c_float), ("bg", C.c_float * 3), ("tile", C.c_int32),
                ("chunk", C.c_int32), ("reorder_k", C.c_int32), ("flags", C.c_uint32),
                ("replay_cap", C.c_int32), ("sort_prefix", C.c_int32)]


class sof_render_out(C.Structure):
    _fields_ = [("color", C.c_void_p), ("depth", C.c_void_p), ("exact_depth", C.c_void_p),
                ("median_depth", C.c_void_p), ("normal", C.c_void_p), ("opacity", C.c_void_p),
                ("n_contrib", C.c_void_p), ("distortion", C.c_void_p), ("extent", C.c_void_p),
                ("opacity_at_depth", C.c_void_p)]


class sof_render_grad_in(C.Structure):
    _fields_ = [("d_color", C.c_void_p), ("d_depth", C.c_void_p), ("d_exact_depth", C.c_void_p),
                ("d_median_depth", C.c_void_p), ("d_normal", C.c_void_p), ("d_opacity", C.c_void_p),
                ("d_distortion", C.c_void_p), ("d_extent", C.c_void_p), ("d_opacity_at_depth", C.c_void_p)]


class sof_scene_grad(C.Structure):
    _fields_ = [("d_means", C.c_void_p), ("d_log_scales", C.c_void_p), ("d_quats", C.c_void_p),
                ("d_opacity_logits", C.c_void_p), ("d_sh", C.c_void_p)]


class sof_query_opts(C.Structure):
    _fields_ = [("near_plane", C.c_float), ("t_stop_query", C.c_float), ("tile", C.c_int32), ("flags", C.c_uint32)]


class sof_stats(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_visible", C.c_int64), ("inexact_pixels", C.c_int64),
                ("nonfinite", C.c_int64), ("n_point_views", C.c_int64), ("n_tests", C.c_int64),
                ("n_hits", C.c_int64), ("n_composited", C.c_int64), ("n_forced", C.c_int64),
                ("n_below_key", C.c_int64), ("n_unsorted", C.c_int64), ("n_replayed", C.c_int64),
                ("n_dropped", C.c_int64), ("n_open", C.c_int64), ("n_read", C.c_int64)]


# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "sof_version": (C.c_int, []),
    "sof_kernel_launches": (C.c_int64, []),
    "sof_error_string": (C.c_char_p, [C.c_int]),
    "sof_last_cuda_error": (C.c_char_p, [C.c_void_p]),
    "sof_workspace_create": (C.c_int, [C.POINTER(C.c_void_p)]),
    "sof_workspace_destroy": (C.c_int, [C.c_void_p]),
    "sof_workspace_bind": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "sof_workspace_required": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "sof_workspace_stats": (C.c_int, [C.c_void_p, C.POINTER(sof_stats)]),
    "sof_workspace_set_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "sof_workspace_clear_dropped": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sof_workspace_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "sof_render_workspace_size": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int,
                                            C.POINTER(sof_render_opts), C.c_int64, C.POINTER(C.c_size_t)]),
    "sof_query_workspace_size": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int, C.c_int64,
                                           C.POINTER(sof_query_opts), C.c_int64, C.POINTER(C.c_size_t)]),
    "sof_render_fwd": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int, C.POINTER(sof_render_opts),
                                 C.POINTER(sof_render_out), C.c_void_p, C.c_void_p]),
    "sof_render_bwd": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int, C.POINTER(sof_render_opts),
                                 C.POINTER(sof_render_out), C.POINTER(sof_render_grad_in), C.POINTER(sof_scene_grad),
                                 C.c_void_p, C.c_void_p]),
    "sof_render_fwd_noalloc": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int,
                                         C.POINTER(sof_render_opts), C.POINTER(sof_render_out),
                                         C.POINTER(C.c_size_t), C.c_void_p]),
    "sof_workspace_reserve": (C.c_int, [C.c_void_p, C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int,
                                        C.POINTER(sof_render_opts), C.c_void_p, C.POINTER(C.c_size_t)]),
    "sof_graph_capture": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int, C.c_int,
                                    C.POINTER(sof_render_opts), C.POINTER(sof_render_out),
                                    C.POINTER(sof_render_grad_in), C.POINTER(sof_scene_grad), C.c_int, C.c_void_p,
                                    C.c_void_p, C.POINTER(C.c_void_p)]),
    "sof_graph_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sof_graph_destroy": (C.c_int, [C.c_void_p]),
    "sof_autotune_candidate": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sof_autotune": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int, C.c_int,
                               C.POINTER(sof_render_opts), C.POINTER(sof_render_out), C.POINTER(sof_render_grad_in),
                               C.POINTER(sof_scene_grad), C.c_int, C.c_char_p, C.c_void_p, C.c_void_p,
                               C.POINTER(sof_render_opts), C.POINTER(C.c_float)]),
    "sof_noalloc_last_error": (C.c_char_p, []),
    "sof_query_prepare": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int, C.c_int64,
                                    C.POINTER(sof_query_opts), C.c_void_p, C.c_void_p]),
    "sof_measure_issue_peaks": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p]),
    "sof_opacity_query": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int, C.c_void_p, C.c_int64,
                                    C.POINTER(sof_query_opts), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sof_level_set_bisect": (C.c_int, [C.POINTER(sof_scene), C.POINTER(sof_camera), C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_int64, C.c_int, C.POINTER(sof_query_opts), C.c_void_p, C.c_void_p]),
}

_lib = None


class SOFError(RuntimeError):
    def __init__(self, code, what, detail=""):
        self.code = code
        super().__init__(f"{what}: {code} ({error_string(code)}) {detail}".strip())


def load():
    """Load libsof.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2506_19139_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def error_string(code: int) -> str:
    try:
        return load().sof_error_string(code).decode()
    except Exception:
        return str(code)


def check(code: int, what: str, ws=None):
    if code < 0:
        detail = ""
        if ws is not None:
            detail = load().sof_last_cuda_error(ws).decode()
        raise SOFError(code, what, detail)
    return code


# --------------------------------------------------------------------------- same-name wrappers

def sof_kernel_launches() -> int:
    return int(load().sof_kernel_launches())


def sof_workspace_create():
    h = C.c_void_p()
    check(load().sof_workspace_create(C.byref(h)), "sof_workspace_create")
    return h


def sof_workspace_destroy(ws):
    return load().sof_workspace_destroy(ws)


def sof_workspace_bind(ws, ptr: int, nbytes: int):
    return check(load().sof_workspace_bind(ws, C.c_void_p(ptr), nbytes), "sof_workspace_bind")


def sof_workspace_required(ws) -> int:
    v = C.c_size_t()
    check(load().sof_workspace_required(ws, C.byref(v)), "sof_workspace_required")
    return int(v.value)


def sof_workspace_stats(ws) -> dict:
    st = sof_stats()
    check(load().sof_workspace_stats(ws, C.byref(st)), "sof_workspace_stats", ws)
    return {k: int(getattr(st, k)) for k, _ in sof_stats._fields_}


# phase indices of sof_workspace_timing (enum in sof.h)
PHASES = ("preprocess", "bin_count", "scan", "bin_emit", "sort", "composite", "fallback", "replay_bwd",
          "composite_bwd", "grad_reduce", "preprocess_bwd", "query_points", "query_integrate")


def sof_workspace_clear_dropped(ws, stream) -> None:
    check(load().sof_workspace_clear_dropped(ws, stream), "sof_workspace_clear_dropped", ws)


def sof_workspace_set_timing(ws, enable: bool) -> None:
    check(load().sof_workspace_set_timing(ws, 1 if enable else 0), "sof_workspace_set_timing", ws)


def sof_workspace_timing(ws) -> dict:
    """{phase: (milliseconds, timed launches)} summed since timing was enabled or last read."""
    ms = (C.c_double * len(PHASES))()
    n = (C.c_int64 * len(PHASES))()
    check(load().sof_workspace_timing(ws, ms, n), "sof_workspace_timing", ws)
    return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(PHASES)}


def sof_render_workspace_size(scene, cams, n_views, opts, pair_capacity) -> int:
    v = C.c_size_t()
    check(load().sof_render_workspace_size(C.byref(scene), cams, n_views, C.byref(opts), pair_capacity, C.byref(v)),
          "sof_render_workspace_size")
    return int(v.value)


def sof_render_fwd(scene, cams, n_views, opts, out, ws, stream) -> int:
    return load().sof_render_fwd(C.byref(scene), cams, n_views, C.byref(opts), C.byref(out), ws, C.c_void_p(stream))


def sof_render_fwd_noalloc(scene, cams, n_views, opts, out, stream):
    """Forward render using the library's fixed device scratch (no allocation). Returns
    (status, required_bytes)."""
    req = C.c_size_t(0)
    rc = load().sof_render_fwd_noalloc(C.byref(scene), cams, n_views, C.byref(opts), C.byref(out), C.byref(req),
                                       C.c_void_p(stream))
    return rc, int(req.value)


def sof_render_bwd(scene, cams, n_views, opts, fwd, gin, grad, ws, stream) -> int:
    return load().sof_render_bwd(C.byref(scene), cams, n_views, C.byref(opts), C.byref(fwd), C.byref(gin),
                                 C.byref(grad), ws, C.c_void_p(stream))


def sof_query_workspace_size(scene, cams, n_views, n_points, opts, pair_capacity) -> int:
    v = C.c_size_t()
    check(load().sof_query_workspace_size(C.byref(scene), cams, n_views, n_points, C.byref(opts), pair_capacity,
                                          C.byref(v)), "sof_query_workspace_size")
    return int(v.value)


def sof_opacity_query(scene, cams, n_views, points, n_points, opts, opacity_out, seen, ws, stream) -> int:
    return load().sof_opacity_query(C.byref(scene), cams, n_views, C.c_void_p(points), n_points, C.byref(opts),
                                    C.c_void_p(opacity_out), C.c_void_p(seen), ws, C.c_void_p(stream))


def sof_level_set_bisect(scene, cams, n_views, inside, outside, n_edges, iterations, opts, ws, stream) -> int:
    return load().sof_level_set_bisect(C.byref(scene), cams, n_views, C.c_void_p(inside), C.c_void_p(outside),
                                       n_edges, iterations, C.byref(opts), ws, C.c_void_p(stream))


def sof_workspace_reserve(ws, scene, cams, n_views, opts, stream) -> tuple:
    """(status, bytes): the workspace size a stream-ordered render of this scene and these views
    needs (synchronises the stream)."""
    b = C.c_size_t(0)
    rc = load().sof_workspace_reserve(ws, C.byref(scene), cams, n_views, C.byref(opts), C.c_void_p(stream),
                                      C.byref(b))
    return rc, int(b.value)


def sof_graph_capture(scene, cams, n_views, views_per_call, opts, out, gin, grad, zero_grads, ws, stream) -> tuple:
    """(status, graph handle or None)."""
    g = C.c_void_p()
    rc = load().sof_graph_capture(C.byref(scene), cams, n_views, views_per_call, C.byref(opts), C.byref(out),
                                  C.byref(gin), C.byref(grad), 1 if zero_grads else 0, ws, C.c_void_p(stream),
                                  C.byref(g))
    return rc, (g if rc == SOF_OK else None)


def sof_graph_launch(graph, stream) -> int:
    return load().sof_graph_launch(graph, C.c_void_p(stream))


def sof_graph_destroy(graph) -> int:
    return load().sof_graph_destroy(graph)


def sof_autotune_candidate(i) -> tuple:
    t, c, k = C.c_int(), C.c_int(), C.c_int()
    check(load().sof_autotune_candidate(i, C.byref(t), C.byref(c), C.byref(k)), "sof_autotune_candidate")
    return int(t.value), int(c.value), int(k.value)


def sof_autotune(scene, cams, n_views, views_per_call, base, out, gin, grad, reps, cache_path, ws, stream) -> tuple:
    """(status, best sof_render_opts, [ms per candidate, -1 where refused])."""
    best = sof_render_opts()
    ms = (C.c_float * SOF_AUTOTUNE_CANDIDATES)()
    rc = load().sof_autotune(C.byref(scene), cams, n_views, views_per_call, C.byref(base), C.byref(out), C.byref(gin),
                             C.byref(grad), reps, cache_path.encode() if cache_path else None, ws, C.c_void_p(stream),
                             C.byref(best), ms)
    return rc, best, [float(x) for x in ms]


def sof_noalloc_last_error() -> str:
    return load().sof_noalloc_last_error().decode()


def sof_measure_issue_peaks(stream=0) -> tuple:
    """(FP32 FMA issue rate, MUFU ex2 rate) of the current device in T op/s, from timed chains."""
    a, b = C.c_double(), C.c_double()
    check(load().sof_measure_issue_peaks(C.byref(a), C.byref(b), C.c_void_p(stream)), "sof_measure_issue_peaks")
    return float(a.value), float(b.value)


def sof_query_prepare(scene, cams, n_views, max_points, opts, ws, stream) -> int:
    return load().sof_query_prepare(C.byref(scene), cams, n_views, max_points, C.byref(opts), ws, C.c_void_p(stream))
