"""The oracle's pins catch plausible mistakes: each case plants one mistake in a copy of the
oracle's C source (a dropped term, a wrong sign or index, a transposed rotation, a wrong weight or
threshold), builds it on the CPU and runs the pins of tests/test_oracle_pins.py against it; at
least one pin must fail. The unmodified source, built the same way, must pass them all.

The copies are built and loaded through SOF_ORACLE_SRC / SOF_ORACLE_LIB, in a child process, so
the oracle that the other tests load is never touched.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sof_oracle.c")

# (name, text in sof_oracle.c, replacement); the first occurrence is the exact-order render's
MUTATIONS = [
    ("2A for 4A in m = C - B^2/4A (Eq. 10)",
     "double m = C - B * B / (4.0 * A);         /* exponent of Eq. 10 */",
     "double m = C - B * B / (2.0 * A);         /* exponent of Eq. 10 */"),
    ("stop decided on T instead of the next T'",
     "                if (Tn < t_stop) {",
     "                if (T < t_stop) {"),
    ("near-plane test dropped",
     "const int inc = alpha >= ALPHA_MIN && tstar > near_plane;",
     "const int inc = alpha >= ALPHA_MIN;"),
    ("crossing value from T' instead of T_k",
     "double gval = (T - 0.5) / (T * G->o);",
     "double gval = (Tn - 0.5) / (T * G->o);"),
    ("normal flipped away from the camera",
     "if (dotv > 0.0) for (int i = 0; i < 3; ++i) G->n[i] = -G->n[i];",
     "if (dotv < 0.0) for (int i = 0; i < 3; ++i) G->n[i] = -G->n[i];"),
    ("E^2 constant 256 for 255 (Eq. 3)",
     "2.0 * log(255.0 * G->o)",
     "2.0 * log(256.0 * G->o)"),
    ("ties broken against the Gaussian index",
     "return (x->g > y->g) - (x->g < y->g);",
     "return (x->g < y->g) - (x->g > y->g);"),
    ("background weighted by 1 - T",
     "color[ip * 3 + i] = Cc[i] + T * (bg ? bg[i] : 0.0);",
     "color[ip * 3 + i] = Cc[i] + (1.0 - T) * (bg ? bg[i] : 0.0);"),
    ("colour and normal weighted by alpha, T dropped",
     "{ Cc[i] += w * G->rgb[i]; Nn[i] += w * G->n[i]; }",
     "{ Cc[i] += h->alpha * G->rgb[i]; Nn[i] += h->alpha * G->n[i]; }"),
    ("depth weighted by alpha, T dropped",
     "D += w * h->t;",
     "D += h->alpha * h->t;"),
    ("sign of one degree-2 SH basis function",
     "Y[5] = -0.5 * sqrt(15.0 / pi) * y * z;",
     "Y[5] = 0.5 * sqrt(15.0 / pi) * y * z;"),
    ("rotation transposed (w negated in the off-diagonal terms)",
     "R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);",
     "R[0][1] = 2 * (x * y + w * z);     R[0][2] = 2 * (x * z - w * y);"),
    ("query evaluated at t* instead of t_eval = min(t*, t) (Eq. 11)",
     "double te = tstar < t ? tstar : t;",
     "double te = tstar;"),
    ("view visibility with W and H swapped",
     "vis = X >= 0.0 && X < cam->W && Y >= 0.0 && Y < cam->H;",
     "vis = X >= 0.0 && X < cam->H && Y >= 0.0 && Y < cam->W;"),
    ("view visibility without the near plane",
     "            if (xc[2] > near_plane) {",
     "            if (xc[2] > 0.0) {"),
    ("interval of results: an ambiguous inclusion taken one way only",
     "        if (!forced && h->amb) {",
     "        if (0) {"),
    ("interval of results: an ambiguous stop taken one way only",
     "            if (!amb_stop || c->over) return;",
     "            return;"),
    ("interval of results: near ties in one order only",
     "            if (k + 1 < c->nh && b_tie(c, k, k + 1)) {",
     "            if (0) {"),
    ("interval of results: an ambiguous crossing taken one way only",
     "            if (!s.pend_cross && s.T > 0.5 && fabs(Tn - 0.5) < c->m_cross * 0.5) {",
     "            if (0) {"),
]


def _run_pins(tmp_path, source_text, tag):
    src = tmp_path / f"oracle_{tag}.c"
    src.write_text(source_text)
    env = dict(os.environ, SOF_ORACLE_SRC=str(src), SOF_ORACLE_LIB=str(tmp_path / f"liboracle_{tag}.so"),
               CUDA_VISIBLE_DEVICES="")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                          capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)


def test_unmodified_copy_passes_the_pins(tmp_path):
    with open(SRC) as f:
        text = f.read()
    r = _run_pins(tmp_path, text, "control")
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_a_pin_catches_the_planted_mistake(tmp_path, name, old, new):
    with open(SRC) as f:
        text = f.read()
    assert old in text, f"mutation site not found: {old}"
    r = _run_pins(tmp_path, text.replace(old, new, 1), "mutant")
    assert r.returncode == 1, f"no pin failed for: {name}\n{r.stdout[-3000:]}"
