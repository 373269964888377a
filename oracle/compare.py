"""Comparison of another implementation's RTCUR result with the FP64 oracle's.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference leg may import or run this module. It imports nothing from the CUDA side.

The support of S^(k) = HT_{zeta_k}(X - L^(k-1)) (Sec. 3.2, Eq. (HT), strict >) is compared entry
by entry. A difference can have two legitimate causes, and each is counted apart:
  * in band:     ||X - L_or^(k-1)| - zeta_k| <= band_rel * zeta_k: the entry sits on the threshold
                 tie within the reported band (1e-6 zeta by default);
  * L-explained: outside the band, but the other implementation's L^(k-1) differs from the
                 oracle's at that entry by at least the entry's distance to the threshold, so its
                 (correct to its precision) |X - L^(k-1)| lies on the other side of zeta.
Every other difference is "unexplained": a wrong support, which parity tests require to be 0.
"""
from __future__ import annotations

import numpy as np

from . import rtcur_oracle as O

__all__ = ["support_flips", "rel_fro", "merge_flips", "entry_groups", "sampled_coords",
           "oracle_values", "compare_entries"]


def rel_fro(a, b):
    """||a - b||_F / ||b||_F (1 as the denominator when b = 0)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


def support_flips(X, S_other, Lprev_other, Lprev_oracle, zeta, band_rel=1e-6, extra=0.0):
    """Support differences of S_other against the oracle's HT_zeta(X - Lprev_oracle) at the same
    entries (arrays of equal shape: X, the other S^(k), the other and the oracle's L^(k-1)).
    ``extra`` widens the L-explained test by an absolute evaluation error of the other side's L
    (a reduced-precision form of the threshold pass evaluates L^(k-1) itself, to about
    2^-16 max|L| in a BF16 split and 2^-11 max|L| in TF32).
    Returns a dict of counts: entries, oracle nonzeros, differences, in band, L-explained and
    unexplained (the last three add up to the differences)."""
    X = np.asarray(X, dtype=np.float64)
    Lo = np.asarray(Lprev_oracle, dtype=np.float64)
    D = X - Lo
    keep_or = np.abs(D) > zeta
    keep_other = np.asarray(S_other) != 0
    diff = keep_or != keep_other
    dist = np.abs(np.abs(D) - zeta)
    inband = diff & (dist <= band_rel * zeta)
    dL = np.abs(np.asarray(Lprev_other, dtype=np.float64) - Lo)
    explained = diff & ~inband & (dist <= dL + extra)
    return {"entries": int(X.size), "nnz_oracle": int(np.count_nonzero(keep_or)),
            "flips": int(np.count_nonzero(diff)), "inband": int(np.count_nonzero(inband)),
            "L_explained": int(np.count_nonzero(explained)),
            "unexplained": int(np.count_nonzero(diff & ~inband & ~explained))}


def merge_flips(parts):
    """Sum the counts of several support_flips results (disjoint groups of entries)."""
    out = {}
    for p in parts:
        for k, v in p.items():
            out[k] = out.get(k, 0) + v
    return out


def entry_groups(dims, seed=1234, n_grid=100, n_slabs=4):
    """Entries at which a large result is compared with the oracle's Tucker state, as index-set
    groups (one index array per mode; a group is their Cartesian product): a seeded random
    n_grid^n grid, then n_slabs seeded whole mode-1 slabs."""
    rng = np.random.default_rng(seed)
    groups = [[np.sort(rng.choice(int(d), size=min(int(d), n_grid), replace=False)) for d in dims]]
    for s in np.sort(rng.choice(int(dims[0]), size=min(int(dims[0]), n_slabs), replace=False)):
        groups.append([np.array([s])] + [np.arange(int(d)) for d in dims[1:]])
    return groups


def sampled_coords(dims, sets):
    """Coordinate arrays (one per mode) of the entries an iteration samples with index sets
    ``sets``: the subtensor R, then the fibers of C_1..C_n (Sec. 3.3)."""
    out = [np.meshgrid(*sets["I"], indexing="ij")]
    for i in range(len(dims)):
        out.append([np.asarray(c) for c in O.fiber_coords(dims, i, sets["J"][i])])
    return out


def oracle_values(ref, dims, last_set, groups):
    """The oracle's L^(k) at the last iteration's sampled entries and at ``groups``, and its
    L^(k-1) at ``groups``, from the Tucker states of an ``rtcur`` result (no full tensor)."""
    st, prev = ref["state"], ref["prev_state"]
    L_sample = [st.eval_subtensor(last_set["I"]).ravel()]
    for i in range(len(dims)):
        L_sample.append(st.eval_fibers(dims, i, last_set["J"][i]).ravel())
    return {"L_sample": np.concatenate(L_sample),
            "L_groups": [O.tucker_eval_subtensor(st.core, st.factors, G) for G in groups],
            "Lprev_groups": [prev.eval_subtensor(G) for G in groups]}


def compare_entries(X, groups, orc, L_sample, L_groups, S_groups, Lprev_groups, zeta, band_rel=1e-6,
                    extra=0.0):
    """Relative Frobenius error of another implementation's L^(k) over the sampled entries and the
    groups, and the support flips of its S^(k) on the groups (merged counts)."""
    Lg = np.concatenate([np.asarray(L_sample, dtype=np.float64).ravel()] +
                        [np.asarray(v, dtype=np.float64).ravel() for v in L_groups])
    Lo = np.concatenate([orc["L_sample"]] + [v.ravel() for v in orc["L_groups"]])
    flips = [support_flips(X[np.ix_(*G)], S_groups[j], Lprev_groups[j], orc["Lprev_groups"][j], zeta,
                           band_rel, extra) for j, G in enumerate(groups)]
    return rel_fro(Lg, Lo), merge_flips(flips)
