"""Writes tests/golden/tiny_scene.json: a tiny seeded scene, one camera and a few query points,
with the FP64 oracle's render (Eq. 1 compositing of Eq. 6-10 peak responses in exact t* order,
Sec. 3.2 exact depth) and opacity field (Eqs. 11-12, App. A.2) of them.

The paper prints no worked example, so these values are the oracle's, computed by this script,
which calls only oracle/ and the seeded input generator. The inputs are stored with the values, so
the fixture does not depend on the generator. Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2506_19139_gb300 import synthetic as syn  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_scene.json")
RENDER_KEYS = ("color", "depth", "exact_depth", "opacity", "normal", "n_contrib", "flags", "slack_color",
               "slack_depth", "slack_normal")


def _f32(a):
    return [float(x) for x in np.asarray(a, np.float32).reshape(-1)]


def main():
    scene = syn.uniform_box_scene(60, 21, 1.0, (0.05, 0.3), (0.1, 0.99), 1)
    cam = syn.look_at((0.4, 0.3, 3.5), (0.0, 0.0, 0.0), 20, 14, 55.0)  # two ragged 16-pixel tiles
    rng = np.random.default_rng(22)
    pts = np.concatenate([scene.means[:6], rng.uniform(-1.0, 1.0, (10, 3))]).astype(np.float32)
    r = oracle.render(scene, cam)
    q = oracle.query(scene, [cam], pts)
    doc = {
        "about": "FP64 oracle render and opacity field of a tiny seeded scene; written by "
                 "tests/golden/make_golden.py (oracle/ only). Render: Eq. 1 over Eq. 6-10 peak responses "
                 "in exact t* order, exact depth of Sec. 3.2; query: Eqs. 11-12 (App. A.2). "
                 "Flags mark pixels or points within a decision margin (several correct results).",
        "scene": {"means": _f32(scene.means), "log_scales": _f32(scene.log_scales), "quats": _f32(scene.quats),
                  "opacity_logits": _f32(scene.opacity_logits), "sh": _f32(scene.sh), "sh_degree": scene.sh_degree,
                  "n": scene.n},
        "camera": {"world_to_cam": _f32(cam.world_to_cam), "fx": float(cam.fx), "fy": float(cam.fy),
                   "cx": float(cam.cx), "cy": float(cam.cy), "width": cam.width, "height": cam.height},
        "render": {k: {"shape": list(np.shape(r[k])), "data": np.asarray(r[k]).reshape(-1).tolist()}
                   for k in RENDER_KEYS},
        "query": {"points": _f32(pts), "opacity": q["opacity"].tolist(), "lo": q["lo"].tolist(),
                  "hi": q["hi"].tolist(), "seen": q["seen"].astype(int).tolist(),
                  "maybe_seen": q["maybe_seen"].astype(int).tolist()},
    }
    with open(OUT, "w") as f:
        json.dump(doc, f)
        f.write("\n")
    print(OUT)


def load():
    """The fixture's scene, camera and points as generator objects, its render (arrays shaped like
    oracle.render's images) and its query values."""
    with open(OUT) as f:
        doc = json.load(f)
    s = doc["scene"]
    n, k = s["n"], (s["sh_degree"] + 1) ** 2
    scene = syn.Scene(np.array(s["means"], np.float32).reshape(n, 3), np.array(s["log_scales"], np.float32).reshape(n, 3),
                      np.array(s["quats"], np.float32).reshape(n, 4), np.array(s["opacity_logits"], np.float32),
                      np.array(s["sh"], np.float32).reshape(n, k, 3), s["sh_degree"])
    c = doc["camera"]
    cam = syn.Camera(np.array(c["world_to_cam"], np.float32).reshape(3, 4), c["fx"], c["fy"], c["cx"], c["cy"],
                     c["width"], c["height"])
    pts = np.array(doc["query"]["points"], np.float32).reshape(-1, 3)
    ref = {k: np.array(v["data"]).reshape(v["shape"]) for k, v in doc["render"].items()}
    for k in ("n_contrib", "flags"):
        ref[k] = ref[k].astype(np.int32)
    return scene, cam, pts, ref, {k: np.array(v) for k, v in doc["query"].items()}


if __name__ == "__main__":
    main()
