"""The stored values of tests/golden/tiny_scene.json are what the oracle computes now. The file was
written by tests/golden/make_golden.py, which calls only the oracle (the paper prints no worked
example to store instead), so a change to the oracle's arithmetic shows here first. It must then
name, in its commit message, the passage or the reading that justifies it."""
import os
import sys

import numpy as np

import oracle

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402


def test_oracle_reproduces_the_stored_render_and_query():
    scene, cam, pts, ref, q = make_golden.load()
    r = oracle.render(scene, cam)
    for k, v in ref.items():
        np.testing.assert_allclose(r[k], v, rtol=1e-12, atol=1e-12, err_msg=k)
    assert (ref["opacity"] > 0).mean() > 0.5  # the fixture is not empty
    o = oracle.query(scene, [cam], pts)
    for k in ("opacity", "lo", "hi"):
        np.testing.assert_allclose(o[k], q[k], rtol=1e-12, atol=1e-12, err_msg=k)
    np.testing.assert_array_equal(o["seen"], q["seen"])
    np.testing.assert_array_equal(o["maybe_seen"], q["maybe_seen"])
