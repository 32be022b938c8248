"""The CUDA path against the stored oracle values of tests/golden/tiny_scene.json (a tiny seeded
scene over two ragged 16-pixel tiles, and 16 query points), without running the oracle: colour,
opacity and normal within 1e-5 absolute, depth within 1e-4 relative (plus a 1e-5 weight error at
the mean ray distance), exact depth within 1e-4 relative, hit counts exact; every query value within
1e-5 of the oracle's interval of correct results. No pixel of the fixture lies within a decision
margin (its flags are all 0)."""
import os
import sys

import numpy as np
import pytest
import torch

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2506_19139_gb300 import build
    build.build()


def test_cuda_render_and_query_match_the_stored_values():
    from paper_2506_19139_gb300 import render as R
    scene, cam, pts, ref, q = make_golden.load()
    assert not ref["flags"].any()
    ts = R.scene_tensors(scene)
    with torch.no_grad():
        res = R.render(*ts, [cam], R.RenderOptions())
        img = {k: v.cpu().numpy().astype(np.float64) for k, v in R.view_images(res, [cam])[0].items()
               if v is not None}
    for k in ("color", "opacity", "normal"):
        err = np.abs(img[k] - ref[k]).max()
        assert err <= 1e-5, f"{k}: {err:.2e}"
    D, O = ref["depth"], ref["opacity"]
    assert np.all(np.abs(img["depth"] - D) <= 1e-4 * np.abs(D) + 1e-5 * D / np.maximum(O, 1e-6) + 1e-7)
    ex = ref["exact_depth"]
    assert np.all(np.abs(img["exact_depth"] - ex) <= 1e-4 * np.abs(ex) + 1e-7)
    np.testing.assert_array_equal(img["n_contrib"].astype(np.int64), ref["n_contrib"])
    o, seen = R.opacity_query(ts[0], ts[1], ts[2], ts[3], [cam], torch.as_tensor(pts, device="cuda"),
                              R.QueryOptions(), R.Workspace())
    torch.cuda.synchronize()
    o = o.cpu().numpy().astype(np.float64)
    assert np.all(o >= q["lo"] - 1e-5) and np.all(o <= q["hi"] + 1e-5), np.abs(o - q["opacity"]).max()
    if seen is not None:
        np.testing.assert_array_equal(seen.cpu().numpy(), q["seen"])
