"""Pins of the comparison module that every parity test and the bench use to judge another
implementation's S^(k) and L^(k) against the oracle (test infrastructure itself, checked here on
hand-built cases whose classification follows from the definitions by inspection)."""
import numpy as np

from oracle import compare as CMP
from oracle import rtcur_oracle as O


def test_support_flips_classifies_each_case():
    zeta = 1.0
    # entries: X, oracle L^(k-1), other L^(k-1), other S^(k) (nonzero = kept)
    # 0: both keep (|X - L| = 2 > 1)                       -> no difference
    # 1: both drop (|X - L| = 0.5)                         -> no difference
    # 2: on the threshold within the band (|X - L| = 1 + 5e-7), other drops -> in band
    # 3: |X - L_or| = 1.01 (oracle keeps), other drops; the other's L differs by 0.02 -> L-explained
    # 4: |X - L_or| = 1.5 (oracle keeps), other drops; the other's L differs by 0.01 -> unexplained
    # 5: |X - L_or| = 0.9 (oracle drops), other keeps; L differs by 0.2 -> L-explained
    # 6: |X - L| = 1 exactly: strict > drops it; other keeps, same L -> in band (distance 0)
    X = np.array([3.0, 1.5, 2.0 + 5e-7, 2.01, 2.5, 1.9, 2.0])
    Lo = np.ones(7)
    Lother = Lo + np.array([0.0, 0.0, 0.0, 0.02, 0.01, 0.2, 0.0])
    S_other = np.array([2.0, 0.0, 0.0, 0.0, 0.0, 0.9, 1.0])
    f = CMP.support_flips(X, S_other, Lother, Lo, zeta)
    assert f == {"entries": 7, "nnz_oracle": 4, "flips": 5, "inband": 2, "L_explained": 2,
                 "unexplained": 1}
    # the evaluation-error allowance of a reduced-precision form explains entry 4 too
    g = CMP.support_flips(X, S_other, Lother, Lo, zeta, extra=0.5)
    assert g["unexplained"] == 0 and g["L_explained"] == 3
    # a tighter band moves entry 2 out of the band; its L does not explain it
    h = CMP.support_flips(X, S_other, Lother, Lo, zeta, band_rel=1e-7)
    assert h["inband"] == 1 and h["unexplained"] == 2


def test_merge_flips_sums_counts():
    a = {"entries": 3, "flips": 1, "inband": 1}
    b = {"entries": 5, "flips": 2, "inband": 0}
    assert CMP.merge_flips([a, b]) == {"entries": 8, "flips": 3, "inband": 1}


def test_rel_fro():
    assert CMP.rel_fro([3.0, 4.0], [3.0, 4.0]) == 0.0
    assert abs(CMP.rel_fro([3.0, 5.0], [3.0, 4.0]) - 0.2) < 1e-15
    assert CMP.rel_fro([1.0, 0.0], [0.0, 0.0]) == 1.0  # zero reference: absolute norm


def test_entry_groups_are_seeded_sorted_and_in_range():
    dims = (30, 20, 25)
    g1 = CMP.entry_groups(dims, seed=5, n_grid=10, n_slabs=3)
    g2 = CMP.entry_groups(dims, seed=5, n_grid=10, n_slabs=3)
    assert len(g1) == 4
    for G1, G2 in zip(g1, g2):
        for a, b, d in zip(G1, G2, dims):
            np.testing.assert_array_equal(a, b)
            assert a.min() >= 0 and a.max() < d and np.all(np.diff(a) > 0)
    assert [len(a) for a in g1[0]] == [10, 10, 10]
    for G in g1[1:]:  # whole mode-1 slabs
        assert len(G[0]) == 1 and len(G[1]) == 20 and len(G[2]) == 25


def test_sampled_coords_cover_the_subtensor_and_the_fibers():
    dims = (6, 5, 7)
    sets = {"I": [np.array([0, 2]), np.array([1, 3, 4]), np.array([5])],
            "J": [np.array([0, 8]), np.array([3]), np.array([1, 2, 4])]}
    cs = CMP.sampled_coords(dims, sets)
    R = cs[0]
    assert R[0].shape == (2, 3, 1)
    assert set(zip(R[0].ravel(), R[1].ravel(), R[2].ravel())) == {
        (a, b, c) for a in (0, 2) for b in (1, 3, 4) for c in (5,)}
    for i in range(3):
        C = cs[1 + i]
        pts = list(zip(*[np.asarray(c).ravel() for c in C]))
        assert len(pts) == dims[i] * len(sets["J"][i])
        # every coordinate of mode i runs through all of 0..d_i - 1 along each fiber
        assert sorted(set(p[i] for p in pts)) == list(range(dims[i]))
        for p in pts:
            assert all(0 <= p[l] < dims[l] for l in range(3))
    # the fibers are those the oracle samples
    for i in range(3):
        ref = O.fiber_coords(dims, i, sets["J"][i])
        for a, b in zip(cs[1 + i], ref):
            np.testing.assert_array_equal(np.asarray(a), np.asarray(b))
