"""Pins of the adjoint oracle (oracle/rtcur_adjoint.py) against things other than itself:
central finite differences in FP64 (masks frozen), the closed form of a linear map, torch's
autograd through its own SVD (an independent derivation of the truncated-pinv derivative), and
consistency with the forward oracle."""
import numpy as np
import pytest

from oracle import rtcur_adjoint as AD
from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import synth


def _fd(f, x, v, h):
    return (f(x + h * v) - f(x - h * v)) / (2.0 * h)


def test_pinv_vjp_matches_central_differences():
    rng = np.random.default_rng(11)
    m, q, r = 7, 11, 3
    # a matrix with a clear gap after sigma_r but not exactly rank r
    U, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((q, q)))
    s = np.array([5.0, 3.0, 2.0, 0.4, 0.2, 0.1, 0.05])
    W = (U * s) @ V[:, :m].T
    for t in range(4):
        Pbar = rng.standard_normal((q, m))
        dW = rng.standard_normal((m, q))
        f = lambda w: float(np.sum(Pbar * O.truncated_pinv(w, r)))
        fd = _fd(f, W, dW, 1e-6)
        an = float(np.sum(AD.pinv_vjp(W, r, Pbar) * dW))
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (t, fd, an)


def test_pinv_vjp_matches_torch_autograd_through_svd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    m, q, r = 6, 9, 2
    W = rng.standard_normal((m, q))
    Pbar = rng.standard_normal((q, m))
    Wt = torch.tensor(W, dtype=torch.float64, requires_grad=True)
    Uu, S, Vh = torch.linalg.svd(Wt, full_matrices=False)
    P = (Vh[:r].T / S[:r]) @ Uu[:, :r].T
    (P * torch.tensor(Pbar)).sum().backward()
    np.testing.assert_allclose(AD.pinv_vjp(W, r, Pbar), Wt.grad.numpy(), rtol=1e-9, atol=1e-10)


def test_tucker_vjp_is_the_adjoint_of_a_linear_map():
    # L is linear in the core: <Lbar, L(core)> = <core_bar, core> exactly
    rng = np.random.default_rng(13)
    core = rng.standard_normal((3, 2, 4))
    F = [rng.standard_normal((5, 3)), rng.standard_normal((6, 2)), rng.standard_normal((4, 4))]
    Lbar = rng.standard_normal((5, 6, 4))
    cb, Fb = AD.tucker_vjp(core, F, Lbar)
    L = O.tucker_full(core, F)
    assert abs(np.sum(Lbar * L) - np.sum(cb * core)) < 1e-10
    # and linear in each factor separately
    for i in range(3):
        assert abs(np.sum(Lbar * L) - np.sum(Fb[i] * F[i])) < 1e-10


def test_fiber_z_reproduces_the_fiber_evaluation():
    rng = np.random.default_rng(14)
    dims = (6, 5, 7)
    R = rng.standard_normal((3, 2, 4))
    A = [rng.standard_normal((6, 3)), rng.standard_normal((5, 2)), rng.standard_normal((7, 4))]
    for i in range(3):
        J = np.sort(rng.choice(int(np.prod(dims)) // dims[i], 5, replace=False))
        np.testing.assert_allclose(A[i] @ AD.fiber_z(R, A, dims, i, J),
                                   O.tucker_eval_fibers(R, A, dims, i, J), rtol=1e-13, atol=1e-13)


def _small_problem(seed=3):
    p = synth.make_tucker_problem((14, 12, 10), (2, 2, 2), 0.2, 3.0, seed=seed, keep_truth=True)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=seed)
    return p, sets


def test_frozen_forward_reproduces_the_oracle():
    p, sets = _small_problem()
    K = 4
    L, tape = AD.frozen_forward(p.X, p.ranks, sets, p.zeta0, p.gamma, K)
    out = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, 0.0, K, keep_full=True)
    np.testing.assert_allclose(L, out["L"], rtol=1e-12, atol=1e-12)
    # replaying the recorded masks gives the same L
    L2, _ = AD.frozen_forward(p.X, p.ranks, sets, p.zeta0, p.gamma, K,
                              masks=[(t["mR"], t["mC"]) for t in tape])
    np.testing.assert_allclose(L2, L, rtol=0, atol=0)


@pytest.mark.parametrize("K", [1, 3])
def test_rtcur_vjp_matches_central_differences(K):
    p, sets = _small_problem(seed=4)
    X = p.X.astype(np.float64)
    L, tape = AD.frozen_forward(X, p.ranks, sets, p.zeta0, p.gamma, K)
    masks = [(t["mR"], t["mC"]) for t in tape]
    Lstar = p.L_star
    dL = 2.0 * (L - Lstar)
    dX = AD.rtcur_vjp(X, tape, p.ranks, dL)
    loss = lambda x: float(np.sum((AD.frozen_forward(x, p.ranks, sets, p.zeta0, p.gamma, K,
                                                     masks=masks)[0] - Lstar) ** 2))
    rng = np.random.default_rng(40 + K)
    for t in range(5):
        v = rng.standard_normal(X.shape)
        v /= np.linalg.norm(v)
        fd = _fd(loss, X, v, 1e-5)
        an = float(np.sum(dX * v))
        assert abs(fd - an) <= 1e-6 * max(np.linalg.norm(dX), 1e-12), (t, fd, an)


def test_rtcur_vjp_is_blind_to_masked_entries_after_one_iteration():
    # K = 1: L^(1) depends on X only through the unmasked sampled slots, so the gradient is zero
    # at every masked slot and off the sample
    p, sets = _small_problem(seed=5)
    X = p.X.astype(np.float64)
    L, tape = AD.frozen_forward(X, p.ranks, sets, p.zeta0, p.gamma, 1)
    dX = AD.rtcur_vjp(X, tape, p.ranks, np.ones_like(L))
    onsample = np.zeros(X.shape, dtype=bool)
    I, J = sets[0]["I"], sets[0]["J"]
    onsample[np.ix_(*I)] = True
    for i in range(3):
        onsample[tuple(O.fiber_coords(X.shape, i, J[i]))] = True
    assert np.all(dX[~onsample] == 0.0)
    masked_only = np.zeros(X.shape, dtype=bool)
    masked_only[np.ix_(*I)] |= tape[0]["mR"]
    unmasked = np.zeros(X.shape, dtype=bool)
    unmasked[np.ix_(*I)] |= ~tape[0]["mR"]
    for i in range(3):
        c = tuple(O.fiber_coords(X.shape, i, J[i]))
        masked_only[c] |= tape[0]["mC"][i]
        unmasked[c] |= ~tape[0]["mC"][i]
    assert np.all(dX[masked_only & ~unmasked] == 0.0)
