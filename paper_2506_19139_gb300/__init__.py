"""GB300-native (sm_103a) compositing core of Sorted Opacity Fields (arXiv 2506.19139).

Exact per-pixel depth-ordered front-to-back compositing of 3D-evaluated Gaussians (forward and
backward) and opacity-field queries at points, behind the C-ABI in include/sof.h. Importing the
package loads nothing; `render` and `_lib` load the in-tree CUDA library on first use and raise if it
is missing (there is no CPU fallback).
"""
__all__ = ["build", "render", "synthetic", "_lib"]
