"""The level-set mode of the opacity query and the bisection for the 0.5 level set (Sec. 3.4
"Early Stopping" and the binary search of marching tetrahedra), against the oracle.

- In SOF_QUERY_LEVEL_SET mode only whether O(x) > 0.5 is exact: it must match the oracle for every
  point whose interval of correct results stays clear of 0.5, and the early stop and the pruning
  across views must cut the evaluated (point, Gaussian) pairs.
- The bisection moves one endpoint per step. Where no step of the oracle's bisection decides
  within the margin of 0.5, the GPU endpoints equal the oracle's exactly (both take FP32
  midpoints); elsewhere the bracket still halves every step and stays on the edge.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2506_19139_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_19139_gb300 import build
    build.build()


def _setup():
    scene = syn.uniform_box_scene(500, 31, 1.0, (0.03, 0.25), (0.2, 0.99), 0)
    cams = [syn.look_at((4 * math.sin(a), 0.6 * math.cos(2 * a), 4 * math.cos(a)), (0.0, 0.0, 0.0), 80, 64, 60.0)
            for a in np.linspace(0, 2 * math.pi, 4, endpoint=False)]
    return scene, cams


def _query(scene, cams, pts, level_set):
    from paper_2506_19139_gb300 import render as R
    ts = R.scene_tensors(scene)
    ws = R.Workspace()
    o, _ = R.opacity_query(ts[0], ts[1], ts[2], ts[3], cams, torch.as_tensor(pts, device="cuda"),
                           R.QueryOptions(level_set=level_set), ws)
    torch.cuda.synchronize()
    return o.cpu().numpy(), ws.stats()


def _clear(ref, margin=2e-5):
    return ~(((ref["lo"] <= 0.5 + margin) & (ref["hi"] > 0.5 - margin)) | (ref["maybe_seen"] != 0))


def test_level_set_query_decides_like_the_oracle():
    scene, cams = _setup()
    rng = np.random.default_rng(4)
    pts = np.concatenate([syn.box_corner_points(scene.subset(np.arange(150)), 1.5),
                          rng.uniform(-1.2, 1.2, (1500, 3)).astype(np.float32)])
    lvl, st_lvl = _query(scene, cams, pts, True)
    exact, st_exact = _query(scene, cams, pts, False)
    ref = oracle.query(scene, cams, pts)
    clear = _clear(ref)
    inside_ref = ref["opacity"] > 0.5
    assert clear.mean() > 0.95
    assert 0.1 < inside_ref[clear].mean() < 0.9
    np.testing.assert_array_equal(lvl[clear] > 0.5, inside_ref[clear])
    np.testing.assert_array_equal(exact[clear] > 0.5, inside_ref[clear])
    # early stop at O_v > 0.5 and pruning of points some view left at or below 0.5
    assert st_lvl["n_tests"] < 0.9 * st_exact["n_tests"]


def _edges(scene, cams, n=600, seed=6):
    """Edges between points the oracle places clearly inside (O > 0.6) and clearly outside (O < 0.4)."""
    rng = np.random.default_rng(seed)
    cand = np.concatenate([scene.means, syn.box_corner_points(scene, 2.0),
                           rng.uniform(-1.2, 1.2, (3000, 3)).astype(np.float32)]).astype(np.float32)
    r = oracle.query(scene, cams, cand)
    ins = cand[(r["lo"] > 0.6) & (r["maybe_seen"] == 0)]
    out = cand[(r["hi"] < 0.4) & (r["maybe_seen"] == 0)]
    k = min(n, ins.shape[0], out.shape[0])
    assert k >= 200
    return ins[rng.choice(ins.shape[0], k, replace=False)], out[rng.choice(out.shape[0], k, replace=False)]


@pytest.mark.parametrize("iterations", [8, 3])
def test_bisection_follows_the_oracle(iterations):
    from paper_2506_19139_gb300 import render as R
    scene, cams = _setup()
    a0, b0 = _edges(scene, cams)
    ts = R.scene_tensors(scene)
    a = torch.as_tensor(a0, device="cuda").clone()
    b = torch.as_tensor(b0, device="cuda").clone()
    R.level_set_bisect(ts[0], ts[1], ts[2], ts[3], cams, a, b, iterations)
    torch.cuda.synchronize()
    a, b = a.cpu().numpy(), b.cpu().numpy()
    ra, rb, amb = oracle.level_set_bisect(scene, cams, a0, b0, iterations)
    assert (~amb).mean() > 0.9
    np.testing.assert_array_equal(a[~amb], ra[~amb])
    np.testing.assert_array_equal(b[~amb], rb[~amb])
    # every edge: the bracket halves each step and stays on the original segment
    L0 = np.linalg.norm(b0 - a0, axis=1)
    L = np.linalg.norm(b - a, axis=1)
    np.testing.assert_allclose(L, L0 / 2 ** iterations, rtol=1e-4, atol=1e-6)
    for p in (a, b):
        s = np.einsum("ij,ij->i", p - a0, b0 - a0) / (L0 * L0)
        off = np.linalg.norm(p - a0 - s[:, None] * (b0 - a0), axis=1)
        assert np.all((s > -1e-5) & (s < 1 + 1e-5)) and np.all(off < 1e-5 * (1 + L0))


def test_bisection_without_edges_or_steps_is_a_no_op():
    from paper_2506_19139_gb300 import render as R
    scene, cams = _setup()
    ts = R.scene_tensors(scene)
    a = torch.zeros((0, 3), device="cuda")
    b = torch.zeros((0, 3), device="cuda")
    R.level_set_bisect(ts[0], ts[1], ts[2], ts[3], cams, a, b, 8)
    a0, b0 = _edges(scene, cams, n=200)
    a = torch.as_tensor(a0, device="cuda").clone()
    b = torch.as_tensor(b0, device="cuda").clone()
    R.level_set_bisect(ts[0], ts[1], ts[2], ts[3], cams, a, b, 0)
    np.testing.assert_array_equal(a.cpu().numpy(), a0)
    np.testing.assert_array_equal(b.cpu().numpy(), b0)
