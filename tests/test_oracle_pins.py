"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test pins one passage; together they are chosen so that a dropped term, a wrong sign,
a wrong index or a transposed operand anywhere in the oracle fails at least one of them."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


def _exact_tucker(dims, ranks, seed):
    L, core, facs = synth.tucker_lowrank(dims, ranks, _rng(seed))
    return L


def _brute_tucker(core, factors):
    """Tucker product by explicit loops over every index (tiny sizes only)."""
    dims = [F.shape[0] for F in factors]
    out = np.zeros(dims)
    for p in itertools.product(*[range(d) for d in dims]):
        s = 0.0
        for c in itertools.product(*[range(r) for r in core.shape]):
            t = core[c]
            for l, F in enumerate(factors):
                t *= F[p[l], c[l]]
            s += t
        out[p] = s
    return out


# ---------------------------------------------------------------- Sec. 2.1 definitions
def test_unfold_columns_are_fibers_in_row_major_order():
    X = np.arange(2 * 3 * 4, dtype=np.float64).reshape(2, 3, 4)
    for i in range(3):
        U = O.unfold(X, i)
        others = [l for l in range(3) if l != i]
        assert U.shape == (X.shape[i], X.size // X.shape[i])
        for j, pc in enumerate(itertools.product(*[range(X.shape[l]) for l in others])):
            for t in range(X.shape[i]):
                p = [0, 0, 0]
                p[i] = t
                for l, v in zip(others, pc):
                    p[l] = v
                assert U[t, j] == X[tuple(p)]
        assert np.array_equal(O.fold(U, i, X.shape), X)


def test_mode_product_matches_index_definition():
    rng = _rng(1)
    X = rng.standard_normal((3, 4, 5))
    for k in range(3):
        A = rng.standard_normal((2, X.shape[k]))
        Y = O.mode_product(X, A, k)
        ref = np.zeros(Y.shape)
        for p in itertools.product(*[range(s) for s in Y.shape]):
            for s in range(X.shape[k]):
                src = list(p)
                src[k] = s
                ref[p] += X[tuple(src)] * A[p[k], s]
        np.testing.assert_allclose(Y, ref, rtol=1e-13, atol=1e-13)


def test_tucker_full_matches_brute_force():
    rng = _rng(2)
    core = rng.standard_normal((2, 3, 2))
    facs = [rng.standard_normal((3, 2)), rng.standard_normal((4, 3)), rng.standard_normal((2, 2))]
    np.testing.assert_allclose(O.tucker_full(core, facs), _brute_tucker(core, facs), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- Sec. 3.2 hard thresholding
def test_hard_threshold_golden_with_ties():
    rows = np.loadtxt(os.path.join(GOLDEN, "ht_small.txt"))
    np.testing.assert_array_equal(O.hard_threshold(rows[:, 0], 2.0), rows[:, 1])


def test_hard_threshold_brute_force_tensor():
    rng = _rng(3)
    D = rng.integers(-4, 5, size=(3, 4, 5)).astype(np.float64)   # many exact ties at zeta = 2
    S = O.hard_threshold(D, 2.0)
    for p in itertools.product(*[range(s) for s in D.shape]):
        assert S[p] == (D[p] if abs(D[p]) > 2.0 else 0.0)


def test_support_property_with_oracle_threshold():
    # Sec. 3.2: zeta = ||L* - L||_inf  =>  supp S subset supp S*, ||S* - S||_inf <= 2 zeta
    rng = _rng(4)
    dims, ranks = (12, 10, 9), (2, 2, 2)
    Ls = _exact_tucker(dims, ranks, 5)
    Ss = synth.planted_outliers(dims, 0.2, 10 * np.mean(np.abs(Ls)), rng, dtype=np.float64)
    X = Ls + Ss
    for scale in (1e-3, 1e-1, 1.0):
        L = Ls + scale * rng.standard_normal(dims)
        zeta = np.max(np.abs(Ls - L))
        S = O.hard_threshold(X - L, zeta)
        assert np.all((S != 0) <= (Ss != 0))
        assert np.max(np.abs(Ss - S)) <= 2 * zeta * (1 + 1e-12)


# ---------------------------------------------------------------- sampled positions
def test_subtensor_and_fiber_evaluation_match_full_tensor():
    rng = _rng(6)
    dims = (5, 6, 4)
    core = rng.standard_normal((2, 3, 2))
    facs = [rng.standard_normal((d, r)) for d, r in zip(dims, core.shape)]
    Lf = O.tucker_full(core, facs)
    I = [np.array([0, 2, 4]), np.array([1, 5]), np.array([0, 1, 3])]
    np.testing.assert_allclose(O.tucker_eval_subtensor(core, facs, I), Lf[np.ix_(*I)], rtol=1e-13, atol=1e-13)
    for i in range(3):
        ncols = int(np.prod(dims)) // dims[i]
        J = np.sort(rng.choice(ncols, size=4, replace=False))
        ref = O.unfold(Lf, i)[:, J]
        np.testing.assert_allclose(O.tucker_eval_fibers(core, facs, dims, i, J), ref, rtol=1e-13, atol=1e-13)
        np.testing.assert_array_equal(O.gather_fibers(Lf, i, J), ref)


def test_fiber_evaluation_four_modes():
    rng = _rng(7)
    dims = (3, 4, 2, 5)
    core = rng.standard_normal((2, 2, 2, 3))
    facs = [rng.standard_normal((d, r)) for d, r in zip(dims, core.shape)]
    Lf = O.tucker_full(core, facs)
    for i in range(4):
        J = np.array([0, 3, int(np.prod(dims)) // dims[i] - 1])
        np.testing.assert_allclose(O.tucker_eval_fibers(core, facs, dims, i, J), O.unfold(Lf, i)[:, J], rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------- SVD_r and the pseudoinverse
def test_truncated_pinv_closed_form():
    rng = _rng(8)
    m, q, r = 7, 11, 3
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    V, _ = np.linalg.qr(rng.standard_normal((q, m)))
    s = np.array([9.0, 5.0, 2.5, 1.0, 0.5, 0.25, 0.1])
    W = Q @ np.diag(s) @ V.T
    expect = V[:, :r] @ np.diag(1.0 / s[:r]) @ Q[:, :r].T        # built from the definition
    np.testing.assert_allclose(O.truncated_pinv(W, r), expect, rtol=1e-11, atol=1e-12)
    # singular values at or below max(m,q) * 2^-24 * s_1 are dropped even when r asks for them
    s2 = s.copy()
    s2[2:] = [1e-7, 1e-9, 0, 0, 0]
    W2 = Q @ np.diag(s2) @ V.T
    expect2 = V[:, :2] @ np.diag(1.0 / s2[:2]) @ Q[:, :2].T
    np.testing.assert_allclose(O.truncated_pinv(W2, 4), expect2, rtol=1e-10, atol=1e-12)
    Qr, sr, Vr = O.svd_truncated(W2, 4)
    assert sr.size == 2


def test_projector_identity():
    # A_i(I_i,:) = W (SVD_r W)^+ = Q_r Q_r^T: symmetric, idempotent, trace r
    rng = _rng(9)
    C = rng.standard_normal((30, 12))
    I = np.sort(rng.choice(30, size=8, replace=False))
    A = C @ O.truncated_pinv(C[I], 3)
    P = A[I]
    np.testing.assert_allclose(P, P.T, atol=1e-12)
    np.testing.assert_allclose(P @ P, P, atol=1e-12)
    assert abs(np.trace(P) - 3) < 1e-12


# ---------------------------------------------------------------- Sec. 2.2 Fiber CUR theorem
def test_fiber_cur_golden_rank1():
    lines = {}
    with open(os.path.join(GOLDEN, "fiber_cur_rank1.txt")) as f:
        for ln in f:
            if ln.startswith("#") or not ln.strip():
                continue
            k, *v = ln.split()
            lines[k] = np.array([float(x) for x in v])
    X = lines["X"].reshape(2, 2, 2)
    I = [np.array([0])] * 3
    J = [np.array([0])] * 3
    R = O.gather_subtensor(X, I)
    C = [O.gather_fibers(X, i, J[i]) for i in range(3)]
    A = O.fiber_cur(R, C, I, (1, 1, 1))
    for i, key in enumerate(("A1", "A2", "A3")):
        np.testing.assert_allclose(A[i][:, 0], lines[key], rtol=1e-15)
    np.testing.assert_allclose(O.tucker_full(R, A), X, rtol=1e-14)


@pytest.mark.parametrize("dims,ranks", [((9, 8, 10), (2, 3, 2)), ((6, 5, 4, 7), (2, 2, 3, 2)), ((12, 15), (3, 3))])
def test_fiber_cur_exact_reconstruction(dims, ranks):
    # Theorem (Sec. 2.2): rank(U_i) = r_i  =>  A = R x_i (C_i U_i^+)
    A_t = _exact_tucker(dims, ranks, 10)
    rng = _rng(11)
    n = len(dims)
    m = [min(d, r + 2) for d, r in zip(dims, ranks)]
    q = [min(int(np.prod(dims)) // dims[i], ranks[i] + 3) for i in range(n)]
    sets = synth.draw_index_set(dims, m, q, rng)
    R = O.gather_subtensor(A_t, sets["I"])
    C = [O.gather_fibers(A_t, i, sets["J"][i]) for i in range(n)]
    for i in range(n):
        assert np.linalg.matrix_rank(C[i][sets["I"][i]]) == ranks[i]
    A = O.fiber_cur(R, C, sets["I"], ranks)
    L = O.tucker_full(R, A)
    assert np.linalg.norm(L - A_t) / np.linalg.norm(A_t) <= 1e-12


def test_truncation_enforces_multilinear_rank():
    # SVD_r in Eq. (R, C_i, U_i): L = R x_i A_i has rank(L_(i)) <= r_i even for full-rank data
    rng = _rng(12)
    X = rng.standard_normal((8, 9, 7))
    sets = synth.draw_index_set(X.shape, [6, 6, 6], [10, 10, 10], rng)
    ranks = (2, 3, 2)
    R = O.gather_subtensor(X, sets["I"])
    C = [O.gather_fibers(X, i, sets["J"][i]) for i in range(3)]
    L = O.tucker_full(R, O.fiber_cur(R, C, sets["I"], ranks))
    for i in range(3):
        s = np.linalg.svd(O.unfold(L, i), compute_uv=False)
        assert np.sum(s > 1e-10 * s[0]) <= ranks[i]


def test_index_order_invariance():
    rng = _rng(13)
    X = rng.standard_normal((8, 7, 6))
    sets = synth.draw_index_set(X.shape, [5, 5, 5], [9, 9, 9], rng)
    ranks = (2, 2, 2)

    def L_of(I, J):
        R = O.gather_subtensor(X, I)
        C = [O.gather_fibers(X, i, J[i]) for i in range(3)]
        return O.tucker_full(R, O.fiber_cur(R, C, I, ranks))

    L0 = L_of(sets["I"], sets["J"])
    I2 = [x[rng.permutation(x.size)] for x in sets["I"]]
    J2 = [x[rng.permutation(x.size)] for x in sets["J"]]
    np.testing.assert_allclose(L_of(I2, J2), L0, rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------- Sec. 3.3 stopping error
def test_relative_error_brute_force():
    rng = _rng(14)
    dims = (5, 4, 6)
    X = rng.standard_normal(dims)
    L = rng.standard_normal(dims)
    S = O.hard_threshold(rng.standard_normal(dims), 1.0)
    sets = synth.draw_index_set(dims, [3, 2, 4], [4, 5, 3], rng)
    E = X - L - S
    num = 0.0
    den = 0.0
    acc_e = sum(E[p] ** 2 for p in itertools.product(*sets["I"]))
    acc_x = sum(X[p] ** 2 for p in itertools.product(*sets["I"]))
    num += math.sqrt(acc_e)
    den += math.sqrt(acc_x)
    for i in range(3):
        coords = O.fiber_coords(dims, i, sets["J"][i])
        acc_e = acc_x = 0.0
        for t in range(dims[i]):
            for b in range(len(sets["J"][i])):
                p = tuple(int(c[t, b]) for c in coords)
                acc_e += E[p] ** 2
                acc_x += X[p] ** 2
        num += math.sqrt(acc_e)
        den += math.sqrt(acc_x)
    ER = O.gather_subtensor(E, sets["I"])
    EC = [O.gather_fibers(E, i, sets["J"][i]) for i in range(3)]
    XR = O.gather_subtensor(X, sets["I"])
    XC = [O.gather_fibers(X, i, sets["J"][i]) for i in range(3)]
    assert abs(O.relative_error(ER, EC, XR, XC) - num / den) <= 1e-14


# ---------------------------------------------------------------- Algorithm 1
def _literal_step(X, L_full, sets, zeta, ranks):
    """One loop body of Algorithm 1 done literally on full tensors (tiny sizes)."""
    S = O.hard_threshold(X - L_full, zeta)
    Y = X - S
    I, J = sets["I"], sets["J"]
    R = Y[np.ix_(*I)]
    C = [O.unfold(Y, i)[:, J[i]] for i in range(X.ndim)]
    A = [C[i] @ O.truncated_pinv(C[i][I[i]], ranks[i]) for i in range(X.ndim)]
    L_new = R
    for i in range(X.ndim):
        L_new = O.mode_product(L_new, A[i], i)
    E = X - L_new - S
    num = np.linalg.norm(E[np.ix_(*I)]) + sum(np.linalg.norm(O.unfold(E, i)[:, J[i]]) for i in range(X.ndim))
    den = np.linalg.norm(X[np.ix_(*I)]) + sum(np.linalg.norm(O.unfold(X, i)[:, J[i]]) for i in range(X.ndim))
    return L_new, num / den


def test_step_matches_literal_algorithm():
    p = synth.make_tucker_problem((10, 9, 8), (2, 2, 2), 0.15, 3, seed=15)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=15)[0]
    X = p.X.astype(np.float64)
    state = O.RTCURState()
    zeta = p.zeta0
    for _ in range(6):
        zeta *= p.gamma
        L_lit, e_lit = _literal_step(X, state.full(p.dims), sets, zeta, p.ranks)
        state, info = O.rtcur_step(X, state, sets, zeta, p.ranks)
        np.testing.assert_allclose(state.full(p.dims), L_lit, rtol=1e-10, atol=1e-10)
        assert abs(info["e"] - e_lit) <= 1e-11


def test_closed_form_single_iteration():
    # S* = 0, exact rank r, zeta0 = 2 max|X|: HT removes nothing, Theorem => L^(1) = X, e^(1) ~ 0
    X = _exact_tucker((14, 12, 10), (3, 2, 3), 16)
    m, q = synth.sample_sizes(X.shape, (3, 2, 3), 3)
    sets = synth.draw_index_sets(X.shape, m, q, seed=16)
    out = O.rtcur(X, (3, 2, 3), sets, 2 * np.max(np.abs(X)), 0.7, 1e-10, 50, "F", keep_full=True)
    assert out["iters"] == 1
    assert out["e"] <= 1e-12
    assert np.linalg.norm(out["L"] - X) / np.linalg.norm(X) <= 1e-12
    assert not np.any(out["S"])


def test_zeta_schedule_and_scope_equivalence():
    p = synth.make_tucker_problem((16, 15, 14), (2, 2, 2), 0.1, 3, seed=17)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=17, n_sets=30)
    a = O.rtcur(p.X, p.ranks, sets, p.zeta0, 0.7, 1e-5, 30, "R", scope="sampled")
    b = O.rtcur(p.X, p.ranks, sets, p.zeta0, 0.7, 1e-5, 30, "R", scope="full")
    z = [p.zeta0]
    for _ in range(a["iters"]):
        z.append(z[-1] * 0.7)
    assert a["hist"]["zeta"] == z[1:]                       # repeated FP64 multiplication
    assert all(x > y for x, y in zip(z, z[1:]))
    assert a["iters"] == b["iters"] and a["hist"]["e"] == b["hist"]["e"]
    np.testing.assert_array_equal(a["state"].core, b["state"].core)


@pytest.mark.parametrize("variant", ["F", "R"])
def test_recovery_of_planted_low_rank(variant):
    # Sec. 4.1 success criterion ||L* - L||_F / ||L*||_F <= 1e-3 at low outlier density
    p = synth.make_tucker_problem((80, 80, 80), (3, 3, 3), 0.1, 3, seed=18)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=18, n_sets=100)
    out = O.rtcur(p.X, p.ranks, sets, p.zeta0, 0.7, 1e-5, 100, variant, keep_full=True)
    assert out["e"] <= 1e-5
    assert np.linalg.norm(out["L"] - p.L_star) / np.linalg.norm(p.L_star) <= 1e-3
    # the found outliers sit on the planted support except near-zero planted values
    S = out["S"]
    assert np.count_nonzero((S != 0) & (p.S_star == 0)) <= 1e-4 * S.size


def test_sample_sizes_golden():
    rows = np.loadtxt(os.path.join(GOLDEN, "sample_sizes.txt"), dtype=np.int64)
    for d1, d2, d3, r, v, m, q in rows:
        mm, qq = synth.sample_sizes((d1, d2, d3), (r, r, r), v)
        assert mm == [m] * 3 and qq == [q] * 3


# --------------------------------------------------------------------------- Chidori form
def test_chidori_sets_give_u_equal_to_unfolded_core():
    # Chidori CUR: J_i = prod_{j != i} I_j, so C_i(I_i, :) is the mode-i unfolding of R (brute force)
    rng = _rng(21)
    for dims, m in (((7, 6, 5), (3, 2, 4)), ((5, 4, 6, 3), (2, 3, 2, 2))):
        X = rng.standard_normal(dims)
        sets = synth.draw_chidori_set(dims, m, rng)
        R = O.gather_subtensor(X, sets["I"])
        for i in range(len(dims)):
            assert np.all(np.diff(sets["J"][i]) > 0) and sets["J"][i].size == np.prod(m) // m[i]
            C = O.gather_fibers(X, i, sets["J"][i])
            np.testing.assert_array_equal(C[sets["I"][i]], O.unfold(R, i))
            # every fiber passes through the core: its other-mode indices lie in their I_j
            for col, jj in enumerate(sets["J"][i][:5]):
                coords = np.unravel_index(jj, [d for k, d in enumerate(dims) if k != i])
                others = [sets["I"][k] for k in range(len(dims)) if k != i]
                assert all(c in o for c, o in zip(coords, others))


@pytest.mark.parametrize("dims,ranks", [((9, 8, 10), (2, 3, 2)), ((6, 5, 4, 7), (2, 2, 3, 2))])
def test_chidori_cur_exact_reconstruction(dims, ranks):
    # rank(U_i) = r_i with the Chidori fibers  =>  R x_i (C_i U_i^+) reproduces the tensor
    A_t = _exact_tucker(dims, ranks, 22)
    rng = _rng(23)
    m = [min(d, r + 2) for d, r in zip(dims, ranks)]
    sets = synth.draw_chidori_set(dims, m, rng)
    R = O.gather_subtensor(A_t, sets["I"])
    C = [O.gather_fibers(A_t, i, sets["J"][i]) for i in range(len(dims))]
    L = O.tucker_full(R, O.fiber_cur(R, C, sets["I"], ranks))
    assert np.linalg.norm(L - A_t) / np.linalg.norm(A_t) <= 1e-12


def test_chidori_recovery_of_planted_low_rank():
    # Sec. 4.1 success criterion with Chidori sampling at low outlier density
    p = synth.make_tucker_problem((30, 30, 30), (2, 2, 2), 0.05, 3.0, seed=24, outlier_scale=1.0,
                                  dtype=np.float64)
    m = [15, 15, 15]
    sets = synth.draw_chidori_sets(p.dims, m, seed=24)
    out = O.rtcur(p.X, p.ranks, sets, float(np.max(np.abs(p.L_star))), 0.7, 1e-5, 100, "F")
    L = out["state"].full(p.dims)
    assert np.linalg.norm(L - p.L_star) / np.linalg.norm(p.L_star) <= 1e-3
