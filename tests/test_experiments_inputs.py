"""The input recipe of the Sec. 4.1 experiment drivers (CPU): the torch generator used on the GPU
also runs on the CPU device, where its output is checked against the recipe itself: exactly
floor(alpha N) corrupted entries, corruption uniform within [-mean|L*|, mean|L*|], L* of
multilinear rank (r, r, r), zeta^(0) = max|L*|, and the same seed giving the same problem."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_tucker_problem_recipe_on_cpu():
    from paper_2108_10448_gb300 import experiments as ex
    d, r, alpha = 24, 3, 0.2
    X, L, z0 = ex.tucker_problem_gpu(d, r, alpha, seed=5, device="cpu")
    X = X.double().numpy()
    L = L.double().numpy()
    S = X - L
    k = int(math.floor(alpha * d ** 3))
    nz = np.abs(S) > 1e-5 * np.abs(L).mean()   # FP32 rounding of X - L elsewhere
    assert int(nz.sum()) == k
    assert np.abs(S[nz]).max() <= np.abs(L).mean() * (1 + 1e-5)
    for i in range(3):  # multilinear rank (r, r, r)
        Li = np.moveaxis(L, i, 0).reshape(d, -1)
        sv = np.linalg.svd(Li, compute_uv=False)
        assert sv[r - 1] > 1e-3 * sv[0] and sv[r] < 1e-5 * sv[0]
    assert z0 == pytest.approx(float(np.abs(L).max()), rel=1e-6)
    X2, L2, _ = ex.tucker_problem_gpu(d, r, alpha, seed=5, device="cpu")
    assert np.array_equal(X2.double().numpy(), X)
