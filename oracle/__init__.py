"""FP64 CPU oracle for the Sorted Opacity Fields compositing core -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import this
package. The product library (paper_2506_19139_gb300) never imports, links or runs it, and the two
share no code: the only common module is the seeded input generator
(paper_2506_19139_gb300.synthetic), which contains no compositing arithmetic.

The C source (sof_oracle.c) follows the paper's definitions directly; see its header for the
passages each function implements. This wrapper only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SOF_ORACLE_SRC lets the mutation test build a copy of the oracle with a planted mistake.
_SRC = os.environ.get("SOF_ORACLE_SRC", os.path.join(_HERE, "sof_oracle.c"))
_LIB = os.environ.get("SOF_ORACLE_LIB", os.path.join(_HERE, "libsof_oracle.so"))
_lock = threading.Lock()
_lib = None

# relative decision margins (alpha vs 1/255, T vs t_stop, t* vs near, t* order, T vs 0.5): a few
# times the FP32 error of the quantity that decides, so that outside them the decision is certain
MARGINS_DEFAULT = np.array([2e-5, 2e-5, 2e-5, 2e-5, 2e-5], dtype=np.float64)
FLAG_ALPHA, FLAG_TSTOP, FLAG_NEAR, FLAG_ORDER, FLAG_CROSS, FLAG_VIEW, FLAG_OVERFLOW = 1, 2, 4, 8, 16, 32, 64
FLAG_EXACT = 128  # exact depth ill-conditioned for FP32 inputs (other outputs unaffected)
FLAG_UNRESOLVED = 256  # more decisions within their margins than the enumeration of results takes
# channels of the interval of correct results (render(..., bounds=True))
BOUND_CHANNELS = ("color0", "color1", "color2", "depth", "normal0", "normal1", "normal2", "opacity", "exact_depth",
                  "n_contrib", "median_depth")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp). Building the checker is not using it."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                                   _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        lib.oracle_render.argtypes = [i64, P, P, P, P, P, i32, P, P, i32, i32, dbl, dbl, P, i32, P, P, i64,
                                      P, P, P, P, P, P, P, P, P, i32, P, P, P, P, i32, P]
        lib.oracle_render_frozen.argtypes = [i64, P, P, P, P, P, i32, P, P, i32, i32, P, P, i64, P, i32, P, P,
                                             P, P, P, P, P, P]
        lib.oracle_render_frozen_f64.argtypes = lib.oracle_render_frozen.argtypes
        lib.oracle_query.argtypes = [i64, P, P, P, P, i32, P, P, P, dbl, dbl, i32, P, P, i64, P, P, P, P, P, P]
        lib.oracle_losses.argtypes = [i64, P, P, P, P, P, P, i32, i32, P, i64, P, i32, P, P]
        lib.oracle_losses_f64.argtypes = lib.oracle_losses.argtypes
        lib.oracle_opa.argtypes = [i64, P, P, P, P, P, P, i32, i32, P, i64, P, i32, P, P]
        lib.oracle_opa_f64.argtypes = lib.oracle_opa.argtypes
        lib.oracle_eval_ray.argtypes = [P, P, P, C.c_float, P, P, P]
        lib.oracle_sh_basis.argtypes = [i32, P, P]
        lib.oracle_gauss_attrs.argtypes = [i64, P, P, P, P, P, i32, P, P, P, P, P, P]
        lib.oracle_num_threads.restype = C.c_int
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _scene_arrays(scene):
    return (_c(scene.means, np.float32), _c(scene.log_scales, np.float32), _c(scene.quats, np.float32),
            _c(scene.opacity_logits, np.float32), _c(scene.sh, np.float32))


def render(scene, cam, near=0.2, t_stop=1e-4, bg=(0.0, 0.0, 0.0), pixels=None, cull=True,
           margins=MARGINS_DEFAULT, max_hits=0, bounds=False, branch_cap=4096):
    """Exact-order FP64 render of one view. Returns a dict of arrays (per selected pixel, or
    images [H,W] / [3,H,W] when pixels is None).

    bounds=True adds "lo" and "hi": per channel of BOUND_CHANNELS the interval of correct results
    (every decision within its margin taken both ways; FLAG_UNRESOLVED where more than branch_cap
    outcomes arise), shaped like the channel's output."""
    lib = _load()
    m, ls, q, lg, sh = _scene_arrays(scene)
    w2c = _c(cam.world_to_cam, np.float32).reshape(-1)
    intr = _c(cam.intr, np.float32)
    W, H = cam.width, cam.height
    pix = None if pixels is None else _c(pixels, np.int64)
    npx = W * H if pix is None else pix.shape[0]
    out = {k: np.zeros(npx, np.float64) for k in ("depth", "exact_depth", "median_depth", "opacity")}
    out["color"] = np.zeros((npx, 3), np.float64)
    out["normal"] = np.zeros((npx, 3), np.float64)
    out["n_contrib"] = np.zeros(npx, np.int32)
    out["flags"] = np.zeros(npx, np.int32)
    hits = np.zeros((npx, max_hits), np.int32) if max_hits > 0 else None
    cross = np.zeros(npx, np.int32)
    delta = np.zeros(npx, np.float64)
    slack = np.zeros((npx, 3), np.float64)
    bgv = _c(bg, np.float64)
    mg = _c(margins, np.float64)
    bnd = np.zeros((npx, 2, len(BOUND_CHANNELS)), np.float64) if bounds else None
    ex_sens = np.zeros(npx, np.float64)
    rc = lib.oracle_render(scene.n, _p(m), _p(ls), _p(q), _p(lg), _p(sh), scene.sh_degree, _p(w2c), _p(intr),
                           W, H, near, t_stop, _p(bgv), int(cull), _p(mg), _p(pix), npx,
                           _p(out["color"]), _p(out["depth"]), _p(out["exact_depth"]), _p(out["median_depth"]),
                           _p(out["normal"]), _p(out["opacity"]), _p(out["n_contrib"]), _p(out["flags"]),
                           _p(hits), max_hits, _p(cross), _p(delta), _p(slack), _p(bnd), int(branch_cap),
                           _p(ex_sens))
    out["overflow"] = bool(rc)
    # how far colour / depth / normal may move under swaps of near-tie hits (both orders correct)
    out["slack_color"], out["slack_depth"], out["slack_normal"] = slack[:, 0], slack[:, 1], slack[:, 2]
    out["hits"] = hits
    # how far FP32-sized relative errors of T_k and m_k move the exact depth (its conditioning)
    out["exact_sens"] = ex_sens
    out["cross_pos"] = cross
    out["delta"] = delta
    if bounds:
        for side, j in (("lo", 0), ("hi", 1)):
            b = bnd[:, j, :]
            out[side] = {"color": b[:, 0:3].copy(), "depth": b[:, 3].copy(), "normal": b[:, 4:7].copy(),
                         "opacity": b[:, 7].copy(), "exact_depth": b[:, 8].copy(), "n_contrib": b[:, 9].copy(),
                         "median_depth": b[:, 10].copy()}
    if pixels is None:
        for k in ("depth", "exact_depth", "median_depth", "opacity", "n_contrib", "flags", "cross_pos", "delta",
                  "slack_color", "slack_depth", "slack_normal", "exact_sens"):
            out[k] = out[k].reshape(H, W)
        out["color"] = out["color"].reshape(H, W, 3).transpose(2, 0, 1).copy()
        out["normal"] = out["normal"].reshape(H, W, 3).transpose(2, 0, 1).copy()
        if bounds:
            for side in ("lo", "hi"):
                d = out[side]
                for k in ("depth", "opacity", "exact_depth", "n_contrib", "median_depth"):
                    d[k] = d[k].reshape(H, W)
                for k in ("color", "normal"):
                    d[k] = d[k].reshape(H, W, 3).transpose(2, 0, 1).copy()
    return out


def render_frozen(scene, cam, hits, cross_pos=None, delta=None, bg=(0.0, 0.0, 0.0), pixels=None):
    """Composite exactly the listed hits per pixel (frozen decisions; detached exact-depth offset
    when delta is given). Outputs per selected pixel, flattened."""
    lib = _load()
    m, ls, q, lg, sh = _scene_arrays(scene)
    w2c = _c(cam.world_to_cam, np.float32).reshape(-1)
    intr = _c(cam.intr, np.float32)
    W, H = cam.width, cam.height
    pix = None if pixels is None else _c(pixels, np.int64)
    npx = W * H if pix is None else pix.shape[0]
    hits = _c(hits, np.int32).reshape(npx, -1)
    cp = None if cross_pos is None else _c(cross_pos, np.int32).reshape(-1)
    dl = None if delta is None else _c(delta, np.float64).reshape(-1)
    out = {k: np.zeros(npx, np.float64) for k in ("depth", "exact_depth", "median_depth", "opacity")}
    out["color"] = np.zeros((npx, 3), np.float64)
    out["normal"] = np.zeros((npx, 3), np.float64)
    bgv = _c(bg, np.float64)
    lib.oracle_render_frozen(scene.n, _p(m), _p(ls), _p(q), _p(lg), _p(sh), scene.sh_degree, _p(w2c), _p(intr),
                             W, H, _p(bgv), _p(pix), npx, _p(hits), hits.shape[1], _p(cp), _p(dl),
                             _p(out["color"]), _p(out["depth"]), _p(out["exact_depth"]), _p(out["median_depth"]),
                             _p(out["normal"]), _p(out["opacity"]))
    return out


def render_frozen_f64(params, sh_degree, cam, hits, cross_pos=None, delta=None, bg=(0.0, 0.0, 0.0),
                      pixels=None):
    """render_frozen with FP64 parameters: params = (means, log_scales, quats, logits, sh) float64."""
    lib = _load()
    m, ls, q, lg, sh = [_c(a, np.float64) for a in params]
    w2c = _c(cam.world_to_cam, np.float32).reshape(-1)
    intr = _c(cam.intr, np.float32)
    W, H = cam.width, cam.height
    pix = None if pixels is None else _c(pixels, np.int64)
    npx = W * H if pix is None else pix.shape[0]
    hits = _c(hits, np.int32).reshape(npx, -1)
    cp = None if cross_pos is None else _c(cross_pos, np.int32).reshape(-1)
    dl = None if delta is None else _c(delta, np.float64).reshape(-1)
    out = {k: np.zeros(npx, np.float64) for k in ("depth", "exact_depth", "median_depth", "opacity")}
    out["color"] = np.zeros((npx, 3), np.float64)
    out["normal"] = np.zeros((npx, 3), np.float64)
    bgv = _c(bg, np.float64)
    lib.oracle_render_frozen_f64(m.shape[0], _p(m), _p(ls), _p(q), _p(lg), _p(sh), sh_degree, _p(w2c), _p(intr),
                                 W, H, _p(bgv), _p(pix), npx, _p(hits), hits.shape[1], _p(cp), _p(dl),
                                 _p(out["color"]), _p(out["depth"]), _p(out["exact_depth"]),
                                 _p(out["median_depth"]), _p(out["normal"]), _p(out["opacity"]))
    return out


NDC_NEAR, NDC_FAR = 0.2, 100.0  # the paper's NDC planes of the distortion and extent losses


def losses(scene, cam, hits, pixels=None, params=None):
    """Distortion and extent losses (Sec. 3.3, App. C.1-C.2) of each pixel over the hits it
    composited, in order (hits as render() returns them). With params (means, log_scales, quats,
    logits as float64 arrays) the Gaussians are taken from there (finite differences)."""
    lib = _load()
    w2c = _c(cam.world_to_cam, np.float32).reshape(-1)
    intr = _c(cam.intr, np.float32)
    W, H = cam.width, cam.height
    pix = None if pixels is None else _c(pixels, np.int64)
    npx = W * H if pix is None else pix.shape[0]
    hits = _c(hits, np.int32).reshape(npx, -1)
    dist = np.zeros(npx, np.float64)
    ext = np.zeros(npx, np.float64)
    if params is None:
        m, ls, q, lg, _ = _scene_arrays(scene)
        fn = lib.oracle_losses
    else:
        m, ls, q, lg = [_c(a, np.float64) for a in params[:4]]
        fn = lib.oracle_losses_f64
    fn(m.shape[0], _p(m), _p(ls), _p(q), _p(lg), _p(w2c), _p(intr), W, H, _p(pix), npx, _p(hits), hits.shape[1],
       _p(dist), _p(ext))
    return {"distortion": dist, "extent": ext}


def opacity_at_depth(scene, cam, hits, exact_depth, pixels=None, params=None):
    """Opacity field at the exact-depth point of each pixel's ray over its composited hits
    (Sec. 3.3, the L_opa supervision); -1 without a 0.5 crossing. exact_depth is taken as given
    (frozen for finite differences); params as in losses()."""
    lib = _load()
    w2c = _c(cam.world_to_cam, np.float32).reshape(-1)
    intr = _c(cam.intr, np.float32)
    W, H = cam.width, cam.height
    pix = None if pixels is None else _c(pixels, np.int64)
    npx = W * H if pix is None else pix.shape[0]
    hits = _c(hits, np.int32).reshape(npx, -1)
    tx = _c(exact_depth, np.float64).reshape(-1)
    out = np.zeros(npx, np.float64)
    if params is None:
        m, ls, q, lg, _ = _scene_arrays(scene)
        fn = lib.oracle_opa
    else:
        m, ls, q, lg = [_c(a, np.float64) for a in params[:4]]
        fn = lib.oracle_opa_f64
    fn(m.shape[0], _p(m), _p(ls), _p(q), _p(lg), _p(w2c), _p(intr), W, H, _p(pix), npx, _p(hits), hits.shape[1],
       _p(tx), _p(out))
    return out


def query(scene, cams, points, near=0.2, t_stop_query=0.0, cull=True, margins=MARGINS_DEFAULT,
          per_view=False):
    """Opacity field at points, min over the views that see each point."""
    lib = _load()
    m, ls, q, lg, _ = _scene_arrays(scene)
    V = len(cams)
    w2c = _c(np.stack([c.world_to_cam.reshape(-1) for c in cams]), np.float32)
    intr = _c(np.stack([c.intr for c in cams]), np.float32)
    wh = _c(np.array([[c.width, c.height] for c in cams]), np.int32)
    pts = _c(points, np.float32).reshape(-1, 3)
    P = pts.shape[0]
    op = np.zeros(P, np.float64)
    seen = np.zeros(P, np.int32)
    flags = np.zeros(P, np.int32)
    pv = np.zeros((P, V), np.float64) if per_view else None
    rng = np.zeros((P, 2), np.float64)
    maybe = np.zeros(P, np.int32)
    mg = _c(margins, np.float64)
    lib.oracle_query(scene.n, _p(m), _p(ls), _p(q), _p(lg), V, _p(w2c), _p(intr), _p(wh), near, t_stop_query,
                     int(cull), _p(mg), _p(pts), P, _p(op), _p(seen), _p(pv), _p(flags), _p(rng), _p(maybe))
    # lo / hi: the interval of correct results when decisions lie within the margins;
    # maybe_seen: views whose visibility of the point is within the margin
    return {"opacity": op, "seen": seen, "flags": flags, "per_view": pv, "lo": rng[:, 0], "hi": rng[:, 1],
            "maybe_seen": maybe}


def level_set_bisect(scene, cams, inside, outside, iterations=8, near=0.2, margin=2e-5):
    """Binary search for the 0.5 level set of O along edges (Sec. 3.4: marching tetrahedra refine
    the surface crossing with 8 bisection steps). Edge e runs from inside[e] (O > 0.5) to
    outside[e] (O <= 0.5). Each step takes the midpoint m = (inside + outside) / 2, rounded to
    FP32 like the points a caller passes, evaluates O(m) with query() and moves inside[e] to m if
    O(m) > 0.5, else outside[e].

    Returns (inside, outside, ambiguous): the final FP32 endpoints and, per edge, whether some step
    decided within the margin of 0.5 (the query's interval of correct results [lo, hi] reaches
    0.5 -/+ margin, or a view's visibility is within its margin), so that either move was correct.
    """
    a = np.array(inside, dtype=np.float32).reshape(-1, 3)
    b = np.array(outside, dtype=np.float32).reshape(-1, 3)
    amb = np.zeros(a.shape[0], dtype=bool)
    for _ in range(iterations):
        m = ((a + b) * np.float32(0.5)).astype(np.float32)
        r = query(scene, cams, m, near=near)
        o = r["opacity"]
        amb |= (r["lo"] <= 0.5 + margin) & (r["hi"] > 0.5 - margin) | (r["maybe_seen"] != 0)
        ins = o > 0.5
        a = np.where(ins[:, None], m, a)
        b = np.where(ins[:, None], b, m)
    return a, b, amb


def eval_ray(mean, log_scale, quat, logit, c, d):
    """A, B, C, t*, m (paper form), m (Gaussian-space cross-product form), o, E^2 for one ray."""
    lib = _load()
    out = np.zeros(8, np.float64)
    lib.oracle_eval_ray(_p(_c(mean, np.float32)), _p(_c(log_scale, np.float32)), _p(_c(quat, np.float32)),
                        C.c_float(float(logit)), _p(_c(c, np.float64)), _p(_c(d, np.float64)), _p(out))
    return dict(zip(("A", "B", "C", "tstar", "m", "m_cross", "o", "E2"), out))


def sh_basis(degree, dirs):
    lib = _load()
    dirs = _c(dirs, np.float64).reshape(-1, 3)
    K = (degree + 1) ** 2
    out = np.zeros((dirs.shape[0], 16), np.float64)
    for i in range(dirs.shape[0]):
        lib.oracle_sh_basis(degree, _p(dirs[i]), C.c_void_p(out.ctypes.data + i * 16 * 8))
    return out[:, :K]


def gauss_attrs(scene, cam):
    lib = _load()
    m, ls, q, lg, sh = _scene_arrays(scene)
    rgb = np.zeros((scene.n, 3)); nrm = np.zeros((scene.n, 3)); op = np.zeros(scene.n); e2 = np.zeros(scene.n)
    lib.oracle_gauss_attrs(scene.n, _p(m), _p(ls), _p(q), _p(lg), _p(sh), scene.sh_degree,
                           _p(_c(cam.world_to_cam, np.float32).reshape(-1)), _p(_c(cam.intr, np.float32)),
                           _p(rgb), _p(nrm), _p(op), _p(e2))
    return {"rgb": rgb, "normal": nrm, "opacity": op, "E2": e2}
