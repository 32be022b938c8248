"""The two gradient references used by the GPU gradient tests agree with each other on CPU:
FP64 central differences of the oracle with frozen decisions, and the independent PyTorch FP64
restatement differentiated by autograd. This pins both before the CUDA backward is checked against them."""
import numpy as np

import test_grad_gpu as G


def test_fd_and_autograd_references_agree():
    scene, cam, ref = G._setup(seed=12, n=60, res=24)
    wts = G._weights(cam, ref["flags"], seed=4)
    fd = G._fd_grads(scene, cam, ref, wts)
    tg, out = G._torch_grads(scene, cam, ref, wts)
    np.testing.assert_allclose(out["color"].detach().numpy(), ref["color"].reshape(3, -1).T, atol=1e-12)
    np.testing.assert_allclose(out["exact_depth"].detach().numpy(), ref["exact_depth"].reshape(-1), atol=1e-12)
    for k in G.GROUPS:
        a, b = tg[k].reshape(-1), fd[k].reshape(-1)
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(b) + 1e-9, k
    assert np.abs(fd["means"]).max() > 0
