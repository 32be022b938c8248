"""Pins of the FP64 oracle against things other than itself (CPU only).

Each check uses an independent route to the value: scipy's quaternion and spherical-harmonic
routines, numeric minimisation of the Mahalanobis distance along a ray, textbook ray/point geometry,
brute force over all Gaussians, and invariants the paper states (App. A.2) or the mathematics
implies. A plausible mistake in the oracle (a dropped term, a wrong sign or index, a transposed
rotation) makes at least one of them fail.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle
from paper_2506_19139_gb300 import synthetic as syn


def _sigma(quat_wxyz, log_scale):
    q = np.asarray(quat_wxyz, dtype=np.float64)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is scalar-last
    s = np.exp(np.asarray(log_scale, dtype=np.float64))
    return R @ np.diag(s * s) @ R.T, R, s


def _mahal(x, mu, Sigma):
    e = x - mu
    return float(e @ np.linalg.solve(Sigma, e))


def _ray_min(mu, Sigma, c, d):
    """Numeric minimum of the Mahalanobis distance along c + t d (Brent)."""
    f = lambda t: _mahal(c + t * d, mu, Sigma)
    t0 = float(np.dot(mu - c, d))
    r = minimize_scalar(f, bracket=(t0 - 0.1, t0 + 0.1), tol=1e-12)
    return r.x, r.fun


def _pixel_ray(cam, px, py):
    R = cam.world_to_cam[:, :3].astype(np.float64)
    t = cam.world_to_cam[:, 3].astype(np.float64)
    c = -R.T @ t
    u = (px + 0.5 - np.float64(np.float32(cam.cx))) / np.float64(np.float32(cam.fx))
    v = (py + 0.5 - np.float64(np.float32(cam.cy))) / np.float64(np.float32(cam.fy))
    d = R.T @ np.array([u, v, 1.0])
    return c, d / np.linalg.norm(d)


def _one(mu, ls, q, logit, rgb=(0.3, 0.6, 0.9)):
    sh = np.zeros((1, 1, 3), np.float32)
    sh[0, 0] = (np.asarray(rgb) - 0.5) / (0.5 / math.sqrt(math.pi))
    return syn.Scene(np.array([mu], np.float32), np.array([ls], np.float32), np.array([q], np.float32),
                     np.array([logit], np.float32), sh, 0)


def _f32(x):
    return np.float64(np.float32(x))


# ----------------------------------------------------------------------------- ray quadratic

def test_isotropic_textbook_geometry():
    """Isotropic Gaussian: t* is the foot of the perpendicular and m = dist^2 / s^2 (no rotation
    convention involved)."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        mu = rng.uniform(-1, 1, 3).astype(np.float32)
        s = rng.uniform(0.02, 0.5)
        ls = np.full(3, math.log(s), np.float32)
        q = rng.standard_normal(4).astype(np.float32)
        c = rng.uniform(-5, 5, 3)
        d = rng.standard_normal(3); d /= np.linalg.norm(d)
        r = oracle.eval_ray(mu, ls, q, 0.3, c, d)
        w = mu.astype(np.float64) - c
        tf = float(np.dot(w, d))
        perp = np.linalg.norm(np.cross(w, d))
        s64 = math.exp(float(ls[0]))
        assert r["tstar"] == pytest.approx(tf, rel=1e-12, abs=1e-12)
        assert r["m"] == pytest.approx(perp ** 2 / s64 ** 2, rel=1e-9, abs=1e-9)
        assert r["A"] == pytest.approx(1.0 / s64 ** 2, rel=1e-12)


def test_anisotropic_matches_numeric_minimum_and_scipy_rotation():
    """Random rotations and scales: A, t*, m agree with Sigma built from scipy's quaternion
    rotation and with a numeric line search; the paper's C - B^2/4A form equals the Gaussian-space
    cross-product form (Eq. 10 vs Eq. 6)."""
    rng = np.random.default_rng(1)
    n_close = 0
    for _ in range(200):
        mu = rng.uniform(-1, 1, 3).astype(np.float32)
        ls = rng.uniform(math.log(0.01), math.log(0.3), 3).astype(np.float32)
        q = rng.standard_normal(4).astype(np.float32)
        Sigma, R, s = _sigma(q, ls)
        c = rng.uniform(-4, 4, 3)
        # aim near the Gaussian so that m is moderate
        target = mu.astype(np.float64) + R @ (s * rng.normal(0, 1.5, 3))
        d = target - c; d /= np.linalg.norm(d)
        r = oracle.eval_ray(mu, ls, q, 0.0, c, d)
        t_num, m_num = _ray_min(mu.astype(np.float64), Sigma, c, d)
        assert r["A"] == pytest.approx(float(d @ np.linalg.solve(Sigma, d)), rel=1e-10)
        assert r["tstar"] == pytest.approx(t_num, rel=1e-7, abs=1e-7)
        assert r["m"] == pytest.approx(m_num, rel=1e-7, abs=1e-9)
        assert r["m_cross"] == pytest.approx(r["m"], rel=1e-9, abs=1e-9)
        n_close += r["m"] < 11.0
    assert n_close > 50


def test_rotation_about_z_moves_local_x_to_world_y():
    """q = (cos 45, 0, 0, sin 45) is a +90 degree turn about z (right-handed): a needle along local x
    becomes a needle along world y."""
    h = math.sqrt(0.5)
    q = np.array([h, 0, 0, h], np.float32)
    ls = np.log(np.array([1.0, 0.01, 0.01], np.float32))
    mu = np.zeros(3, np.float32)
    c = np.array([0.0, 0.0, -5.0])
    # ray parallel to z through (0, 0.5, .): 0.5 along world y is inside the needle (s=1) only if
    # the needle lies along y
    d = np.array([0.0, 0.0, 1.0])
    r_y = oracle.eval_ray(mu, ls, q, 0.0, c + np.array([0.0, 0.5, 0.0]), d)
    r_x = oracle.eval_ray(mu, ls, q, 0.0, c + np.array([0.5, 0.0, 0.0]), d)
    assert r_y["m"] == pytest.approx(0.25, rel=1e-9)
    assert r_x["m"] == pytest.approx(2500.0, rel=1e-6)


def test_opacity_cutoff_radius():
    """E^2 = 2 ln(255 o) (Eq. 3): at Mahalanobis radius E the un-clamped alpha equals 1/255."""
    for o in (0.01, 0.3, 0.99):
        logit = math.log(o / (1 - o))
        r = oracle.eval_ray(np.zeros(3, np.float32), np.zeros(3, np.float32), np.array([1, 0, 0, 0], np.float32),
                            logit, np.array([0.0, 0.0, -3.0]), np.array([0.0, 0.0, 1.0]))
        o32 = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
        assert r["o"] == pytest.approx(o32, rel=1e-12)
        assert o32 * math.exp(-0.5 * r["E2"]) == pytest.approx(1.0 / 255.0, rel=1e-12)


# ----------------------------------------------------------------------------- SH and attributes

def _real_sh_scipy(deg, dirs):
    """Real SH of degree <= deg from scipy's complex SH (Condon-Shortley phase kept):
    m>0: sqrt2 Re Y_l^m, m<0: sqrt2 Im Y_l^|m|, m=0: Y_l^0; ordered m = -l..l."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    cols = []
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                cols.append(math.sqrt(2) * Y.real)
            elif m < 0:
                cols.append(math.sqrt(2) * Y.imag)
            else:
                cols.append(Y.real)
    return np.stack(cols, axis=1)


def test_sh_basis_matches_scipy_and_is_orthonormal():
    rng = np.random.default_rng(2)
    dirs = rng.standard_normal((64, 3)); dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    ours = oracle.sh_basis(3, dirs)
    ref = _real_sh_scipy(3, dirs)
    np.testing.assert_allclose(ours, ref, rtol=1e-12, atol=1e-12)
    # Gauss-Legendre x uniform-phi quadrature is exact for these degree<=6 products
    xg, wg = np.polynomial.legendre.leggauss(12)
    ph = np.linspace(0, 2 * np.pi, 24, endpoint=False)
    Z, PH = np.meshgrid(xg, ph, indexing="ij")
    Wt = np.outer(wg, np.full(ph.size, 2 * np.pi / ph.size)).reshape(-1)
    st = np.sqrt(1 - Z ** 2)
    D = np.stack([(st * np.cos(PH)).reshape(-1), (st * np.sin(PH)).reshape(-1), Z.reshape(-1)], axis=1)
    Y = oracle.sh_basis(3, D)
    gram = (Y * Wt[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_dc_colour_and_normal_reading():
    scene, cams = syn.tiny_forward(0, n=64)
    a = oracle.gauss_attrs(scene, cams[0])
    rgb_drawn = scene.sh[:, 0, :].astype(np.float64) * (0.5 / math.sqrt(math.pi)) + 0.5
    np.testing.assert_allclose(a["rgb"], np.maximum(rgb_drawn, 0), atol=1e-6)
    # normal: unit, along the smallest principal axis (scipy rotation), facing the camera
    Rc = cams[0].world_to_cam[:, :3].astype(np.float64)
    c = -Rc.T @ cams[0].world_to_cam[:, 3].astype(np.float64)
    for g in range(scene.n):
        _, R, s = _sigma(scene.quats[g], scene.log_scales[g])
        axis = R[:, int(np.argmin(s))]
        n = a["normal"][g]
        assert abs(abs(float(np.dot(n, axis))) - 1.0) < 1e-12
        assert float(np.dot(n, scene.means[g].astype(np.float64) - c)) <= 0.0


# ----------------------------------------------------------------------------- render

def _brute_alpha(scene, g, c, d):
    Sigma, _, _ = _sigma(scene.quats[g], scene.log_scales[g])
    t, m = _ray_min(scene.means[g].astype(np.float64), Sigma, c, d)
    o = 1.0 / (1.0 + math.exp(-float(scene.opacity_logits[g])))
    return t, m, min(0.99, o * math.exp(-0.5 * m)), o


def test_single_gaussian_closed_form_all_pixels():
    """One Gaussian: colour = alpha rgb + (1 - alpha) bg, depth = alpha t*, opacity = alpha, with
    alpha from a numeric line search; exact depth solves 1 - o G(t) = 0.5 on the camera side."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 24, 20, 60.0)
    q = np.array([0.9, 0.2, -0.3, 0.1], np.float32)
    ls = np.log(np.array([0.5, 0.3, 0.15], np.float32))
    mu = np.array([0.1, -0.05, 0.2], np.float32)
    logit = math.log(0.9 / 0.1)
    scene = _one(mu, ls, q, logit)
    bg = np.array([0.05, 0.1, 0.2])
    out = oracle.render(scene, cam, bg=bg)
    Sigma, Rg, sg = _sigma(q, ls)
    n_axis = Rg[:, int(np.argmin(sg))]
    if np.dot(n_axis, mu.astype(np.float64) - np.array([0.0, 0.0, 4.0])) > 0:
        n_axis = -n_axis
    rgb = np.array([0.3, 0.6, 0.9])
    n_checked = 0
    for py in range(cam.height):
        for px in range(cam.width):
            c, d = _pixel_ray(cam, px, py)
            t, m, a, o = _brute_alpha(scene, 0, c, d)
            hit = a >= 1 / 255 and t > 0.2 and (1 - a) >= 1e-4
            ae = a if hit else 0.0
            np.testing.assert_allclose(out["color"][:, py, px], ae * rgb + (1 - ae) * bg, atol=1e-9)
            np.testing.assert_allclose(out["normal"][:, py, px], ae * n_axis, atol=1e-9)
            assert out["depth"][py, px] == pytest.approx(ae * t, abs=1e-8)
            assert out["opacity"][py, px] == pytest.approx(ae, abs=1e-10)
            if hit and 1 - a <= 0.5:
                te = out["exact_depth"][py, px]
                assert te <= t + 1e-9
                g = math.exp(-0.5 * _mahal(c + te * d, mu.astype(np.float64), Sigma))
                assert 1.0 - o * g == pytest.approx(0.5, abs=1e-9)
                n_checked += 1
            else:
                assert out["exact_depth"][py, px] == 0.0
    assert n_checked > 10


def test_two_gaussians_front_to_back_order_and_crossing_residual():
    """Two Gaussians on the optical axis: the nearer one is composited first; the exact depth on
    the crossing Gaussian satisfies T_k (1 - o_k G(t)) = 0.5 with T_k from the front one."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 9, 9, 60.0)
    sc_a = _one([0.0, 0.0, 0.6], np.log([0.2, 0.2, 0.2]), [1, 0, 0, 0], math.log(0.35 / 0.65), rgb=(1, 0, 0))
    sc_b = _one([0.02, 0.0, -0.4], np.log([0.3, 0.25, 0.1]), [0.8, 0.1, 0.5, 0.2], math.log(0.95 / 0.05), rgb=(0, 0, 1))
    # put the far one first in memory: order must come from t*, not from the index
    scene = syn.Scene(np.concatenate([sc_b.means, sc_a.means]), np.concatenate([sc_b.log_scales, sc_a.log_scales]),
                      np.concatenate([sc_b.quats, sc_a.quats]), np.concatenate([sc_b.opacity_logits, sc_a.opacity_logits]),
                      np.concatenate([sc_b.sh, sc_a.sh]), 0)
    out = oracle.render(scene, cam, max_hits=4)
    c, d = _pixel_ray(cam, 4, 4)
    tb, mb, ab, ob = _brute_alpha(scene, 0, c, d)
    ta, ma, aa, oa = _brute_alpha(scene, 1, c, d)
    assert ta < tb
    col = out["color"][:, 4, 4]
    np.testing.assert_allclose(col, [aa, 0.0, (1 - aa) * ab], atol=1e-9)
    assert list(out["hits"][4 * 9 + 4][:2]) == [1, 0]
    assert out["depth"][4, 4] == pytest.approx(aa * ta + (1 - aa) * ab * tb, rel=1e-9)
    assert out["opacity"][4, 4] == pytest.approx(1 - (1 - aa) * (1 - ab), abs=1e-12)
    Tk = 1 - aa
    assert Tk > 0.5 and Tk * (1 - ab) < 0.5
    te = out["exact_depth"][4, 4]
    Sigma_b, _, _ = _sigma(scene.quats[0], scene.log_scales[0])
    g = math.exp(-0.5 * _mahal(c + te * d, scene.means[0].astype(np.float64), Sigma_b))
    assert Tk * (1 - ob * g) == pytest.approx(0.5, abs=1e-9)
    assert out["median_depth"][4, 4] == pytest.approx(tb, rel=1e-7)


def test_stop_rule_and_near_plane():
    """Opaque stack on the axis: compositing stops before the hit that drops T below 1e-4; a
    Gaussian whose peak lies closer than the near plane is never composited."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 5, 5, 60.0)
    zs = [1.0, 0.5, 0.0, -0.5, -1.0, 3.9]  # the last is 0.1 in front of the camera
    parts = [_one([0, 0, z], np.log([0.3, 0.3, 0.3]), [1, 0, 0, 0], math.log(0.9 / 0.1), rgb=(1, 1, 1)) for z in zs]
    scene = syn.Scene(*[np.concatenate([getattr(p, k) for p in parts]) for k in
                        ("means", "log_scales", "quats", "opacity_logits", "sh")], 0)
    out = oracle.render(scene, cam, max_hits=8)
    c, d = _pixel_ray(cam, 2, 2)
    alphas = sorted([(_brute_alpha(scene, g, c, d)[0], _brute_alpha(scene, g, c, d)[2], g) for g in range(len(zs))])
    T, used = 1.0, []
    for t, a, g in alphas:
        if t <= 0.2:
            continue
        if T * (1 - a) < 1e-4:
            break
        used.append(g); T *= 1 - a
    assert 5 not in used
    assert out["n_contrib"][2, 2] == len(used) < 5
    assert list(out["hits"][2 * 5 + 2][:len(used)]) == used
    assert out["opacity"][2, 2] == pytest.approx(1 - T, abs=1e-12)
    # the comparison is strict and the hit that crosses the threshold is excluded
    T = 1.0
    for k, (t, a, g) in enumerate([h for h in alphas if h[0] > 0.2][:4]):
        Tn = T * (1 - a)
        above = oracle.render(scene, cam, t_stop=Tn * (1 + 1e-9), pixels=np.array([2 * 5 + 2]))
        below = oracle.render(scene, cam, t_stop=Tn * (1 - 1e-9), pixels=np.array([2 * 5 + 2]))
        assert above["n_contrib"][0] == k
        assert below["n_contrib"][0] >= k + 1
        T = Tn


def test_equal_depth_ties_follow_gaussian_index():
    """Two Gaussians with identical geometry tie exactly in t*: the lower index is composited
    first."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 3, 3, 60.0)
    a = _one([0, 0, 0], np.log([0.3, 0.3, 0.3]), [1, 0, 0, 0], math.log(0.6 / 0.4), rgb=(1, 0, 0))
    b = _one([0, 0, 0], np.log([0.3, 0.3, 0.3]), [1, 0, 0, 0], math.log(0.6 / 0.4), rgb=(0, 1, 0))
    scene = syn.Scene(*[np.concatenate([getattr(a, k), getattr(b, k)]) for k in
                        ("means", "log_scales", "quats", "opacity_logits", "sh")], 0)
    out = oracle.render(scene, cam, max_hits=2)
    al = out["opacity"][1, 1]
    a1 = 1 - math.sqrt(1 - al)
    np.testing.assert_allclose(out["color"][:, 1, 1], [a1, (1 - a1) * a1, 0.0], atol=1e-12)
    assert list(out["hits"][4]) == [0, 1]


def test_culled_equals_brute_force_and_invariants():
    """The culled path equals evaluating every Gaussian at every pixel; sum of weights plus final
    transmittance is 1; permuting the Gaussians changes nothing; 0 <= opacity <= 1."""
    scene, cams = syn.tiny_forward(0, n=300)
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 32, 32, 60.0)
    a = oracle.render(scene, cam, cull=True)
    b = oracle.render(scene, cam, cull=False)
    for k in ("color", "depth", "exact_depth", "normal", "opacity", "n_contrib"):
        np.testing.assert_array_equal(a[k], b[k])
    white = syn.Scene(scene.means, scene.log_scales, scene.quats, scene.opacity_logits,
                      np.full_like(scene.sh, (1.0 - 0.5) / (0.5 / math.sqrt(math.pi))), 0)
    w = oracle.render(white, cam)
    np.testing.assert_allclose(w["color"][0], w["opacity"], atol=1e-12)
    assert (a["opacity"] >= 0).all() and (a["opacity"] <= 1).all()
    perm = np.random.default_rng(5).permutation(scene.n)
    p = oracle.render(scene.subset(perm), cam)
    for k in ("color", "depth", "exact_depth", "normal", "opacity", "n_contrib"):
        np.testing.assert_allclose(a[k], p[k], atol=1e-12)
    assert (a["n_contrib"] > 0).sum() > 100


def test_transmittance_non_increasing_and_frozen_replay():
    """Replaying the recorded hit lists reproduces the render, and truncating the lists gives a
    non-increasing transmittance."""
    scene, cams = syn.tiny_forward(3, n=400)
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 24, 24, 60.0)
    out = oracle.render(scene, cam, max_hits=64)
    assert not out["overflow"]
    fz = oracle.render_frozen(scene, cam, out["hits"], out["cross_pos"].reshape(-1))
    np.testing.assert_allclose(fz["color"], out["color"].reshape(3, -1).T, atol=1e-12)
    np.testing.assert_allclose(fz["exact_depth"], out["exact_depth"].reshape(-1), atol=1e-12)
    prev = np.zeros(cam.width * cam.height)
    for k in range(1, 12):
        h = out["hits"].copy()
        h[:, k:] = -1
        o = oracle.render_frozen(scene, cam, h)["opacity"]
        assert (o >= prev - 1e-15).all()
        prev = o


# ----------------------------------------------------------------------------- opacity field

def test_query_is_one_minus_product_of_brute_force_alphas():
    """O_N(x) = 1 - prod(1 - alpha_i(min(t*_i, t))) (App. A.2), alphas from a numeric line search."""
    rng = np.random.default_rng(7)
    scene = syn.uniform_box_scene(25, 8, 0.6, (0.1, 0.4), (0.2, 0.95), 0)
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 64, 64, 60.0)
    pts = rng.uniform(-0.7, 0.7, (40, 3)).astype(np.float32)
    res = oracle.query(scene, [cam], pts)
    R = cam.world_to_cam[:, :3].astype(np.float64)
    c = -R.T @ cam.world_to_cam[:, 3].astype(np.float64)
    for i, x in enumerate(pts.astype(np.float64)):
        t = np.linalg.norm(x - c); d = (x - c) / t
        P = 1.0
        for g in range(scene.n):
            Sigma, _, _ = _sigma(scene.quats[g], scene.log_scales[g])
            mu = scene.means[g].astype(np.float64)
            ts, _ = _ray_min(mu, Sigma, c, d)
            te = min(ts, t)
            o = 1.0 / (1.0 + math.exp(-float(scene.opacity_logits[g])))
            a = min(0.99, o * math.exp(-0.5 * _mahal(c + te * d, mu, Sigma)))
            if a >= 1 / 255 and ts > 0.2:
                P *= 1 - a
        assert res["seen"][i] == 1
        assert res["opacity"][i] == pytest.approx(1 - P, abs=1e-9)


def test_query_far_point_equals_render_opacity_without_stop():
    """A point far behind every Gaussian on a pixel's ray sees every Gaussian at its peak, so
    O_N equals the render's accumulated opacity with the transmittance stop disabled."""
    scene, _ = syn.tiny_forward(4, n=500)
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 48, 48, 60.0)
    out = oracle.render(scene, cam, t_stop=1e-300)
    pts, pix = [], []
    for py in range(6, 42, 5):
        for px in range(6, 42, 5):
            c, d = _pixel_ray(cam, px, py)
            pts.append(c + 30.0 * d); pix.append((py, px))
    q = oracle.query(scene, [cam], np.array(pts, np.float32))
    for i, (py, px) in enumerate(pix):
        assert q["opacity"][i] == pytest.approx(out["opacity"][py, px], abs=2e-6)


def test_query_at_exact_depth_is_half():
    """Sec. 3.2: for a lone Gaussian the exact depth lies on the 0.5 level set of the opacity
    field, so querying c + t_exact d returns 0.5."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 40, 40, 60.0)
    scene = _one([0.05, -0.02, 0.1], np.log([0.6, 0.5, 0.3]), [0.7, -0.2, 0.4, 0.3], math.log(0.97 / 0.03))
    out = oracle.render(scene, cam)
    pts = []
    for py in range(40):
        for px in range(40):
            te = out["exact_depth"][py, px]
            if te > 0:
                c, d = _pixel_ray(cam, px, py)
                pts.append(c + te * d)
    assert len(pts) > 20
    q = oracle.query(scene, [cam], np.array(pts, np.float32))
    np.testing.assert_allclose(q["opacity"], 0.5, atol=2e-6)


def test_query_min_over_views_and_unseen():
    scene, _ = syn.tiny_forward(5, n=200)
    cams = [syn.look_at((4 * math.sin(a), 0.5, 4 * math.cos(a)), (0, 0, 0), 40, 30, 60.0) for a in (0.0, 2.0, 4.0)]
    pts = np.random.default_rng(9).uniform(-1.2, 1.2, (200, 3)).astype(np.float32)
    pts = np.concatenate([pts, np.array([[50.0, 50.0, 50.0]], np.float32)])
    r = oracle.query(scene, cams, pts, per_view=True)
    pv = r["per_view"]
    for i in range(pts.shape[0]):
        vis = pv[i] >= 0
        assert r["seen"][i] == vis.sum()
        assert r["opacity"][i] == (pv[i][vis].min() if vis.any() else 1.0)
    assert r["seen"][-1] == 0 and r["opacity"][-1] == 1.0
    c = oracle.query(scene, cams, pts, cull=False)
    np.testing.assert_array_equal(c["opacity"], r["opacity"])


# ----------------------------------------------------------------------------- several correct results

def test_near_tie_slack_covers_both_orders():
    """Two hits whose t* differ by less than the order margin may be composited in either order
    (P11). The oracle's slack must be 2 T_a alpha_a alpha_b |c_a - c_b| (closed form of the swap)
    and cover the colour of the other order, evaluated independently by the frozen compositor;
    pairs farther apart get no slack."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 9, 9, 60.0)
    lin = 4 * 9 + 4
    for eps, tie in ((1e-6, True), (1e-3, False)):
        sa = _one([0.0, 0.0, 0.0], np.log([0.3, 0.3, 0.3]), [1, 0, 0, 0], math.log(0.4 / 0.6), rgb=(1, 0.2, 0))
        sb = _one([0.05, 0.0, -eps], np.log([0.25, 0.25, 0.25]), [1, 0, 0, 0], math.log(0.7 / 0.3), rgb=(0, 0.5, 1))
        scene = syn.Scene(np.concatenate([sa.means, sb.means]), np.concatenate([sa.log_scales, sb.log_scales]),
                          np.concatenate([sa.quats, sb.quats]), np.concatenate([sa.opacity_logits, sb.opacity_logits]),
                          np.concatenate([sa.sh, sb.sh]), 0)
        out = oracle.render(scene, cam, max_hits=4)
        c, d = _pixel_ray(cam, 4, 4)
        ta, _, aa, _ = _brute_alpha(scene, 0, c, d)
        tb, _, ab, _ = _brute_alpha(scene, 1, c, d)
        assert ta < tb and (tb - ta) / tb < (2e-6 if tie else 1.0)
        slack = out["slack_color"][4, 4]
        assert bool(out["flags"][4, 4] & oracle.FLAG_ORDER) == tie
        if not tie:
            assert slack == 0.0
            continue
        ca, cb = np.array([1, 0.2, 0]), np.array([0, 0.5, 1])
        assert slack == pytest.approx(2 * aa * ab * np.abs(ca - cb).max(), rel=1e-6)  # FP32 SH colour
        hits = np.full((1, 4), -1, np.int32)
        hits[0, :2] = [1, 0]   # the other order
        sw = oracle.render_frozen(scene, cam, hits, pixels=np.array([lin]))
        assert np.abs(sw["color"][0] - out["color"][:, 4, 4]).max() <= slack
        assert np.abs(sw["color"][0] - out["color"][:, 4, 4]).max() >= 0.4 * slack  # the slack is tight
        assert sw["opacity"][0] == pytest.approx(out["opacity"][4, 4], abs=1e-15)


def test_query_range_covers_an_ambiguous_inclusion():
    """A Gaussian whose alpha at the query point lies within the margin of 1/255 may be included or
    not (P11): the oracle's range must span the opacity of both choices; clear of the margin the
    range collapses to the value."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 16, 16, 60.0)
    c = np.array([0.0, 0.0, 4.0])
    mu = np.array([0.3, 0.0, 0.0])
    x = np.array([0.0, 0.0, -3.0], np.float32)          # on the optical axis, far behind the Gaussian
    d = (x - c) / np.linalg.norm(x - c)
    Sigma, _, _ = _sigma([1, 0, 0, 0], np.log([0.2, 0.2, 0.2]))
    _, m = _ray_min(mu, Sigma, c, d)
    for rel, amb in ((5e-6, True), (1e-2, False)):
        o = (1.0 / 255.0) * (1.0 + rel) * math.exp(0.5 * m)
        sc = _one(mu, np.log([0.2, 0.2, 0.2]), [1, 0, 0, 0], math.log(o / (1 - o)))
        r = oracle.query(sc, [cam], x[None])
        alpha = o * math.exp(-0.5 * m)
        assert r["seen"][0] == 1
        assert bool(r["flags"][0] & oracle.FLAG_ALPHA) == amb
        if amb:
            assert r["lo"][0] <= 1e-12 and r["hi"][0] >= alpha * (1 - 1e-9)
        else:
            assert r["lo"][0] == pytest.approx(alpha, rel=1e-6) and r["hi"][0] == pytest.approx(alpha, rel=1e-6)
        assert r["lo"][0] <= r["opacity"][0] <= r["hi"][0]


def test_level_set_bisection_closed_form_crossing():
    """Sec. 3.4 binary search for the 0.5 level set. On the camera axis through an isotropic
    Gaussian (o = 0.9, s = 0.1) at distance 4, O at distance t < 4 is alpha = o exp(-(t - 4)^2 /
    (2 s^2)), so O = 0.5 at t_c = 4 - s sqrt(2 ln(2 o)). Twenty steps from the centre (inside,
    O = o) to a point 3 in front (outside) bracket t_c within 2^-20 of the edge, with the inside
    end behind the crossing and the outside end in front of it."""
    s, o = 0.1, 0.9
    sc = _one([0.0, 0.0, 0.0], [math.log(s)] * 3, [1.0, 0.0, 0.0, 0.0], math.log(o / (1.0 - o)))
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 32, 32, 60.0)
    t_c = 4.0 - s * math.sqrt(2.0 * math.log(2.0 * o))
    z_c = 4.0 - t_c  # the crossing's z on the axis (the camera looks down -z from z = 4)
    inside = np.array([[0.0, 0.0, 0.0]], np.float32)
    outside = np.array([[0.0, 0.0, 1.0]], np.float32)
    a, b, amb = oracle.level_set_bisect(sc, [cam], inside, outside, iterations=20)
    assert b[0, 2] - a[0, 2] <= 1.0 / 2 ** 20 * 1.0001
    # the ends straddle the crossing (up to FP32 rounding of the coordinates; the last steps decide
    # within the margin of 0.5, which the oracle flags)
    assert a[0, 2] <= z_c + 1e-7 and z_c - 1e-7 <= b[0, 2]
    assert abs(0.5 * (a[0, 2] + b[0, 2]) - z_c) < 1e-6
    r = oracle.query(sc, [cam], np.concatenate([a, b]))
    assert r["opacity"][0] > 0.5 >= r["opacity"][1]
    # eight steps, as in the paper, stay away from the margin here
    a8, b8, amb8 = oracle.level_set_bisect(sc, [cam], inside, outside, iterations=8)
    assert not amb8[0] and a8[0, 2] <= z_c <= b8[0, 2] and b8[0, 2] - a8[0, 2] <= 1.0 / 256 * 1.0001


def _ndc(t):
    return oracle.NDC_FAR * (t - oracle.NDC_NEAR) / ((oracle.NDC_FAR - oracle.NDC_NEAR) * t)


def test_distortion_and_extent_closed_form_on_the_axis():
    """Sec. 3.3 losses on the camera axis through two isotropic Gaussians (peaks at their centres,
    m = 0, alpha = o): distortion = w1 w2 (NDC(t1) - NDC(t2))^2 with w1 = o1, w2 = o2 (1 - o1); the
    extent of a lone Gaussian is near far / (far - near) o s sqrt(2 ln(255 o)) / t^2 (eps = s E)."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 33, 33, 60.0)
    o1, o2, s1, s2 = 0.6, 0.8, 0.05, 0.08
    sc = syn.Scene(np.array([[0.0, 0.0, 1.0], [0.0, 0.0, -1.0]], np.float32),
                   np.log(np.array([[s1] * 3, [s2] * 3], np.float32)),
                   np.array([[1.0, 0.0, 0.0, 0.0]] * 2, np.float32),
                   np.array([math.log(o1 / (1 - o1)), math.log(o2 / (1 - o2))], np.float32),
                   np.zeros((2, 1, 3), np.float32), 0)
    pix = np.array([16 * 33 + 16], np.int64)  # the centre pixel's ray is the axis
    out = oracle.render(sc, cam, pixels=pix, max_hits=4)
    assert list(out["hits"][0][:2]) == [0, 1]
    L = oracle.losses(sc, cam, out["hits"], pixels=pix)
    t1, t2 = 3.0, 5.0
    w1, w2 = _f32(o1), _f32(o2) * (1.0 - _f32(o1))
    assert L["distortion"][0] == pytest.approx(w1 * w2 * (_ndc(t1) - _ndc(t2)) ** 2, rel=1e-6)
    c = oracle.NDC_NEAR * oracle.NDC_FAR / (oracle.NDC_FAR - oracle.NDC_NEAR)
    e = lambda o, s, t: _f32(o) * _f32(s) * math.sqrt(2.0 * math.log(255.0 * _f32(o))) / t ** 2
    assert L["extent"][0] == pytest.approx(c * (w1 / _f32(o1) * e(o1, s1, t1) + w2 / _f32(o2) * e(o2, s2, t2)),
                                           rel=1e-5)
    one = oracle.losses(sc.subset([0]), cam, out["hits"][:, :1], pixels=pix)
    assert one["distortion"][0] == 0.0 and one["extent"][0] == pytest.approx(c * e(o1, s1, t1), rel=1e-5)


def test_distortion_equals_the_prefix_sum_form():
    """App. C.1: sum_i w_i (d_i^2 A_{i-1} + D2_{i-1} - 2 d_i D_{i-1}) (prefix sums of w, w d, w d^2)
    equals the oracle's pair sum, with alpha and t* of each hit from eval_ray's paper-form
    quadratic (an independent route); so does the closed form of the final sums, A D2 - D^2 (half
    the sum over all ordered pairs), which the GPU forward writes."""
    scene, cams = syn.tiny_forward(3)
    cam = cams[0]
    out = oracle.render(scene, cam, max_hits=256)
    L = oracle.losses(scene, cam, out["hits"])
    rng = np.random.default_rng(2)
    cand = np.flatnonzero(out["n_contrib"].reshape(-1) >= 3)
    for ip in rng.choice(cand, 20, replace=False):
        px, py = ip % cam.width, ip // cam.width
        c, d = _pixel_ray(cam, px, py)
        T, A, D, D2, total = 1.0, 0.0, 0.0, 0.0, 0.0
        for g in out["hits"].reshape(cam.width * cam.height, -1)[ip]:
            if g < 0:
                break
            r = oracle.eval_ray(scene.means[g], scene.log_scales[g], scene.quats[g], scene.opacity_logits[g], c, d)
            a = min(0.99, r["o"] * math.exp(-0.5 * r["m"]))
            w = a * T
            dn = _ndc(r["tstar"])
            total += w * (dn * dn * A + D2 - 2.0 * dn * D)
            A, D, D2 = A + w, D + w * dn, D2 + w * dn * dn
            T *= 1.0 - a
        assert L["distortion"].reshape(-1)[ip] == pytest.approx(total, rel=1e-9, abs=1e-15)
        assert L["distortion"].reshape(-1)[ip] == pytest.approx(A * D2 - D * D, rel=1e-7, abs=1e-13)
        assert A == pytest.approx(1.0 - T, rel=1e-12)


def test_opacity_at_depth_equals_the_query_and_one_half_for_a_lone_gaussian():
    """Sec. 3.3 L_opa: the opacity field at the exact-depth point of a pixel's ray, over the
    pixel's composited hits, equals the query of Eqs. 11-12 (all Gaussians, the point's own ray) at
    c + t d wherever the render did not stop early; for a lone Gaussian it is 0.5 (Sec. 3.2)."""
    scene, cams = syn.tiny_forward(0)
    cam = cams[0]
    out = oracle.render(scene, cam, max_hits=256)
    o = oracle.opacity_at_depth(scene, cam, out["hits"], out["exact_depth"])
    ex = out["exact_depth"].reshape(-1)
    stopped = out["opacity"].reshape(-1) > 1.0 - 2e-4
    sel = np.flatnonzero((ex > 0) & ~stopped)
    assert sel.size > 100 and np.all(o[ex <= 0] == -1.0)
    pts = []
    for ip in sel:
        c, d = _pixel_ray(cam, ip % cam.width, ip // cam.width)
        pts.append(c + ex[ip] * d)
    q = oracle.query(scene, [cam], np.array(pts, np.float32))
    np.testing.assert_allclose(o[sel], q["opacity"], atol=2e-5)
    assert (o[sel] < 0.45).mean() > 0.01  # hits in front of the point but past it in t* count less
    lone = _one([0.05, -0.02, 0.1], np.log([0.6, 0.5, 0.3]), [0.7, -0.2, 0.4, 0.3], math.log(0.97 / 0.03))
    cam2 = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 40, 40, 60.0)
    r = oracle.render(lone, cam2, max_hits=4)
    o2 = oracle.opacity_at_depth(lone, cam2, r["hits"], r["exact_depth"])
    assert (o2 >= 0).sum() > 20
    np.testing.assert_allclose(o2[o2 >= 0], 0.5, atol=1e-9)


# ------------------------------------------------------- the interval of correct render results

def _stack(parts):
    return syn.Scene(*[np.concatenate([getattr(p, k) for p in parts]) for k in
                       ("means", "log_scales", "quats", "opacity_logits", "sh")], 0)


def test_render_bounds_take_an_ambiguous_alpha_both_ways():
    """One isotropic Gaussian whose peak alpha on the centre pixel lies within the margin of 1/255
    (P11): the bounds span excluding it (opacity 0, background colour, no hit) and including it
    (alpha from a numeric line search, its colour); clear of the margin they collapse to the value."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 9, 7, 60.0)
    c, d = _pixel_ray(cam, 4, 3)
    mu = np.array([0.25, 0.0, 0.0])
    ls = np.log(np.full(3, 0.2, np.float32)).astype(np.float32)
    Sigma, _, _ = _sigma([1, 0, 0, 0], ls)
    _, m = _ray_min(mu, Sigma, c, d)
    rgb = np.array([0.3, 0.6, 0.9])
    for rel, amb in ((5e-6, True), (-5e-6, True), (1e-2, False)):
        o = (1.0 / 255.0) * (1.0 + rel) * math.exp(0.5 * m)
        sc = _one(mu, ls, [1, 0, 0, 0], math.log(o / (1 - o)))
        o32 = 1.0 / (1.0 + math.exp(-float(sc.opacity_logits[0])))
        alpha = o32 * math.exp(-0.5 * m)
        r = oracle.render(sc, cam, bounds=True, bg=(0.1, 0.1, 0.1), pixels=np.array([3 * 9 + 4]))
        lo, hi = r["lo"], r["hi"]
        assert bool(r["flags"][0] & oracle.FLAG_ALPHA) == amb
        if amb:
            assert lo["opacity"][0] == 0.0 and hi["opacity"][0] == pytest.approx(alpha, rel=1e-9)
            assert lo["n_contrib"][0] == 0 and hi["n_contrib"][0] == 1
            want = alpha * rgb + (1 - alpha) * 0.1
            np.testing.assert_allclose(hi["color"][0], np.maximum(want, 0.1), rtol=1e-9)
            np.testing.assert_allclose(lo["color"][0], np.minimum(want, 0.1), rtol=1e-9)
        else:
            assert lo["opacity"][0] == hi["opacity"][0] == r["opacity"][0] == pytest.approx(alpha, rel=1e-9)


def test_render_bounds_take_an_ambiguous_stop_both_ways():
    """An opaque stack on the axis with t_stop set within the margin of the transmittance after
    hit k: the bounds hold the result that stops before hit k and the one that composites it,
    each computed independently by rendering with t_stop just above / below that transmittance."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 5, 5, 60.0)
    parts = [_one([0, 0, z], np.log([0.3, 0.3, 0.3]), [1, 0, 0, 0], math.log(0.9 / 0.1), rgb=(r, 1 - r, 0.5))
             for z, r in zip([1.0, 0.5, 0.0, -0.5, -1.0], [0.1, 0.9, 0.3, 0.7, 0.5])]
    scene = _stack(parts)
    lin = np.array([2 * 5 + 2])
    full = oracle.render(scene, cam, t_stop=1e-12, pixels=lin, max_hits=8)
    assert full["n_contrib"][0] == 5
    alphas = []
    c, d = _pixel_ray(cam, 2, 2)
    for g in full["hits"][0][:5]:
        alphas.append(_brute_alpha(scene, int(g), c, d)[2])
    T = 1.0
    for k in range(1, 4):
        T *= 1 - alphas[k - 1]
        Tk = T * (1 - alphas[k])  # the transmittance after hit k (0-based)
        r = oracle.render(scene, cam, t_stop=Tk * (1 + 5e-6), pixels=lin, bounds=True)
        assert r["flags"][0] & oracle.FLAG_TSTOP
        stop = oracle.render(scene, cam, t_stop=Tk * (1 + 1e-3), pixels=lin)
        go = oracle.render(scene, cam, t_stop=Tk * (1 - 1e-3), pixels=lin)
        assert stop["n_contrib"][0] == k and go["n_contrib"][0] == k + 1
        for side in (stop, go):
            for ch in ("opacity", "depth", "n_contrib"):
                assert r["lo"][ch][0] <= side[ch][0] + 1e-12 and side[ch][0] <= r["hi"][ch][0] + 1e-12, (k, ch)
            assert np.all(r["lo"]["color"][0] <= side["color"][0] + 1e-12)
            assert np.all(side["color"][0] <= r["hi"]["color"][0] + 1e-12)
        assert r["lo"]["n_contrib"][0] == k and r["hi"]["n_contrib"][0] == k + 1


def test_render_bounds_take_an_ambiguous_near_plane_both_ways():
    """A Gaussian whose peak lies within the margin of the near plane (t* = near (1 +- 5e-6)) may
    be a hit or not: opacity bounds [0, alpha]."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 5, 5, 60.0)
    c, d = _pixel_ray(cam, 2, 2)
    for rel in (5e-6, -5e-6):
        sc = _one([0.0, 0.0, 4.0 - 0.2 * (1 + rel)], np.log([0.05, 0.05, 0.05]), [1, 0, 0, 0], math.log(0.8 / 0.2))
        t, _, a, _ = _brute_alpha(sc, 0, c, d)
        assert abs(t / 0.2 - 1) < 1e-5
        r = oracle.render(sc, cam, pixels=np.array([12]), bounds=True)
        assert r["flags"][0] & oracle.FLAG_NEAR or rel < 0
        assert r["lo"]["opacity"][0] == 0.0 and r["hi"]["opacity"][0] == pytest.approx(a, rel=1e-7)


def test_render_bounds_take_an_ambiguous_crossing_both_ways():
    """A lone Gaussian whose peak alpha is 0.5 (1 - 5e-6): T' = 1 - alpha lies within the margin of
    0.5, so the 0.5 crossing may be found on it or not. Exact depth: 0 (no crossing) or the depth
    where alpha(t) = 0.5, which for a peak just below 0.5 is the peak t* itself."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 5, 5, 60.0)
    c, d = _pixel_ray(cam, 2, 2)
    mu = np.array([0.05, 0.0, 0.0])
    Sigma, _, _ = _sigma([1, 0, 0, 0], np.log([0.2, 0.2, 0.2]))
    t, m = _ray_min(mu, Sigma, c, d)
    o = 0.5 * (1 - 5e-6) * math.exp(0.5 * m)
    sc = _one(mu, np.log([0.2, 0.2, 0.2]), [1, 0, 0, 0], math.log(o / (1 - o)))
    r = oracle.render(sc, cam, pixels=np.array([12]), bounds=True)
    assert r["exact_depth"][0] == 0.0
    assert r["lo"]["exact_depth"][0] == 0.0
    assert r["hi"]["exact_depth"][0] == pytest.approx(t, rel=1e-6)


def test_render_bounds_take_a_near_tie_in_both_orders():
    """Two hits whose t* differ by less than the order margin: the colour bounds are exactly the
    two orders' colours, the other order computed by the frozen compositor."""
    cam = syn.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 9, 9, 60.0)
    lin = 4 * 9 + 4
    sa = _one([0.0, 0.0, 0.0], np.log([0.3, 0.3, 0.3]), [1, 0, 0, 0], math.log(0.4 / 0.6), rgb=(1, 0.2, 0))
    sb = _one([0.05, 0.0, -1e-6], np.log([0.25, 0.25, 0.25]), [1, 0, 0, 0], math.log(0.7 / 0.3), rgb=(0, 0.5, 1))
    scene = _stack([sa, sb])
    r = oracle.render(scene, cam, max_hits=4, bounds=True, pixels=np.array([lin]))
    assert r["flags"][0] & oracle.FLAG_ORDER
    other = np.full((1, 4), -1, np.int32)
    other[0, :2] = r["hits"][0][:2][::-1]
    sw = oracle.render_frozen(scene, cam, other, pixels=np.array([lin]))
    both = np.stack([r["color"][0], sw["color"][0]])
    np.testing.assert_allclose(r["lo"]["color"][0], both.min(axis=0), atol=1e-15)
    np.testing.assert_allclose(r["hi"]["color"][0], both.max(axis=0), atol=1e-15)
    assert np.any(r["hi"]["color"][0] - r["lo"]["color"][0] > 1e-3)


def test_render_bounds_contain_the_fp64_result_and_collapse_without_flags():
    """On random scenes (dense overlap included), every pixel's FP64 result lies in its bounds, and
    pixels with no decision within a margin have bounds equal to it."""
    for scene, cam in ((syn.tiny_forward(0)[0], syn.tiny_forward(0)[1][0]),
                       (syn.uniform_box_scene(400, 9, 0.8, (0.05, 0.5), (0.05, 0.6), 0),
                        syn.look_at((0.0, 0.0, 2.2), (0.0, 0.0, 0.0), 64, 48, 70.0))):
        r = oracle.render(scene, cam, bounds=True)
        F = r["flags"]
        assert not np.any(F & oracle.FLAG_UNRESOLVED)
        clear = (F & (oracle.FLAG_ALPHA | oracle.FLAG_TSTOP | oracle.FLAG_NEAR | oracle.FLAG_ORDER |
                      oracle.FLAG_CROSS)) == 0
        for ch in ("opacity", "depth", "n_contrib", "exact_depth"):
            assert np.all(r["lo"][ch] <= r[ch] + 1e-12) and np.all(r[ch] <= r["hi"][ch] + 1e-12), ch
            assert np.array_equal(r["lo"][ch][clear], r[ch][clear]) and np.array_equal(r["hi"][ch][clear], r[ch][clear])
        for ch in ("color", "normal"):
            assert np.all(r["lo"][ch] <= r[ch] + 1e-12) and np.all(r[ch] <= r["hi"][ch] + 1e-12), ch


# ------------------------------------------------------------------ which views see a point (P12)

def test_query_visibility_rule_against_back_projected_points():
    """P12: a view sees x iff z_cam > near and its projection lies in [0, W) x [0, H). Points are
    made by back-projecting pixel coordinates just inside and just outside each image edge (and
    depths just beyond / short of the near plane) of a non-square image, so a swapped W and H, an
    off-by-one at an edge or a wrong near test changes some answer."""
    W, H = 40, 24
    cam = syn.look_at((0.3, -0.2, 4.0), (0.0, 0.1, 0.0), W, H, 60.0)
    R = cam.world_to_cam[:, :3].astype(np.float64)
    tv = cam.world_to_cam[:, 3].astype(np.float64)
    fx, fy, cx, cy = (np.float64(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))

    def point(X, Y, z):
        pc = np.array([(X - cx) / fx * z, (Y - cy) / fy * z, z])
        return R.T @ (pc - tv)

    e = 1e-2
    cases = []
    for X, Y, want in ((e, H / 2, True), (-e, H / 2, False), (W - e, H / 2, True), (W + e, H / 2, False),
                       (W / 2, e, True), (W / 2, -e, False), (W / 2, H - e, True), (W / 2, H + e, False),
                       (H - e, W - e, False), (W - e, H - e, True), (H + e, H / 2, True), (W / 2, W - 2, False)):
        cases.append((point(X, Y, 3.0), want))
    cases.append((point(W / 2, H / 2, 0.2 * (1 + 1e-3)), True))
    cases.append((point(W / 2, H / 2, 0.2 * (1 - 1e-3)), False))
    pts = np.array([p for p, _ in cases], np.float32)
    empty = _one([50.0, 50.0, 50.0], np.log([0.01, 0.01, 0.01]), [1, 0, 0, 0], -10.0)
    r = oracle.query(empty, [cam], pts)
    for (p, want), got, fl in zip(cases, r["seen"], r["flags"]):
        assert bool(fl & oracle.FLAG_VIEW) is False
        assert bool(got) == want, (p, want)
