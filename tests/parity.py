"""Element-by-element check of the CUDA render against the FP64 oracle's interval of correct results
(shared by the render parity tests; not a test module itself).

Where a decision lies within a margin of its threshold (alpha = 1/255, T' = t_stop, the near plane,
two hits with nearly equal t*, T' = 0.5 at the crossing), several results are correct (P11
reading). oracle.render(..., bounds=True) takes every such decision both ways and returns per pixel
and channel the interval [lo, hi] of the correct results. Every pixel's GPU value must lie inside,
widened by the tolerances:
  colour, opacity, normal: 1e-5 absolute;
  depth (the un-normalised sum of w t*), median depth: 1e-4 relative (+1e-7);
  exact depth: max(1e-4 relative, 2x its predicted FP32 conditioning) (+1e-7);
  hit count: exact.
A pixel is left out only if its decisions need more outcomes than the oracle enumerates
(FLAG_UNRESOLVED); an exact depth is left out only where a crossing decision within its margin makes
it depend on the rounding of T near 0.5 (infinite bounds). Both are counted, printed and bounded.
"""
import numpy as np

import oracle


def flat(gpu):
    """Per-pixel rows of view_images() output: [P] scalars, [P,3] colour and normal."""
    out = {}
    for k, v in gpu.items():
        v = np.asarray(v)
        out[k] = v.reshape(3, -1).T if k in ("color", "normal") else v.reshape(-1)
    return out


def check_bounds(gpu, ref, label, max_unresolved_frac=1e-4, max_exact_undetermined_frac=2e-3, median=False):
    """gpu, ref: per-pixel rows (flat(); ref from oracle.render(..., pixels=..., bounds=True) or
    flattened the same way). Returns {channel: (pixels outside, largest excess)} and the fractions
    left out."""
    F = np.asarray(ref["flags"]).reshape(-1)
    lo = {k: np.asarray(v).reshape(F.size, -1).squeeze(-1) if k not in ("color", "normal") else v
          for k, v in ref["lo"].items()}
    hi = {k: np.asarray(v).reshape(F.size, -1).squeeze(-1) if k not in ("color", "normal") else v
          for k, v in ref["hi"].items()}
    n = F.size
    unres = (F & oracle.FLAG_UNRESOLVED) != 0
    ex_undet = ~(np.isfinite(lo["exact_depth"]) & np.isfinite(hi["exact_depth"])) & ~unres
    frac_unres, frac_undet = float(unres.sum()) / n, float(ex_undet.sum()) / n
    print(f"{label}: {n} pixels, {int((F != 0).sum())} with decisions within a margin, "
          f"{int(unres.sum())} unresolved ({100 * frac_unres:.4f}%), "
          f"{int(ex_undet.sum())} exact depths undetermined ({100 * frac_undet:.4f}%)")
    assert frac_unres <= max_unresolved_frac, f"{label}: {int(unres.sum())} unresolved pixels"
    assert ex_undet.sum() <= max(2, max_exact_undetermined_frac * n), \
        f"{label}: {int(ex_undet.sum())} undetermined exact depths"
    ok = ~unres

    def outside(g, l, h, tol):
        """How far g lies outside [l - tol, h + tol] (<= 0 inside)."""
        with np.errstate(over="ignore", invalid="ignore"):
            return np.maximum(l - tol - g, g - h - tol)

    def mag(k):
        return np.maximum(np.abs(np.nan_to_num(lo[k])), np.abs(np.nan_to_num(hi[k])))

    sens = np.asarray(ref["exact_sens"]).reshape(-1)
    ex_tol = np.maximum(1e-4 * mag("exact_depth"), 2.0 * sens) + 1e-7
    over = {
        "color": outside(gpu["color"], lo["color"], hi["color"], 1e-5).max(axis=1),
        "opacity": outside(gpu["opacity"], lo["opacity"], hi["opacity"], 1e-5),
        "normal": outside(gpu["normal"], lo["normal"], hi["normal"], 1e-5).max(axis=1),
        "depth": outside(gpu["depth"], lo["depth"], hi["depth"], 1e-4 * mag("depth") + 1e-7),
        "exact_depth": np.where(ex_undet, -1.0, outside(gpu["exact_depth"], np.nan_to_num(lo["exact_depth"]),
                                                        np.nan_to_num(hi["exact_depth"]), ex_tol)),
        "n_contrib": outside(gpu["n_contrib"].astype(np.float64), lo["n_contrib"], hi["n_contrib"], 0.0),
    }
    if median:
        over["median_depth"] = outside(gpu["median_depth"], lo["median_depth"], hi["median_depth"],
                                       1e-4 * mag("median_depth") + 1e-7)
    msg = {k: (int((ok & (v > 0)).sum()), float(np.max(np.where(ok, v, -np.inf), initial=-np.inf)))
           for k, v in over.items()}
    for k, v in over.items():
        bad = ok & (v > 0)
        assert not bad.any(), (f"{label}: {k} outside the interval of correct results {msg} "
                               f"at rows {np.argwhere(bad)[:4].ravel().tolist()}")
    return msg, {"unresolved": frac_unres, "exact_undetermined": frac_undet}
