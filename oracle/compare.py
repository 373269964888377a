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

__all__ = ["support_flips", "rel_fro", "merge_flips"]


def rel_fro(a, b):
    """||a - b||_F / ||b||_F (1 as the denominator when b = 0)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b)) / (nb if nb > 0 else 1.0)


def support_flips(X, S_other, Lprev_other, Lprev_oracle, zeta, band_rel=1e-6):
    """Support differences of S_other against the oracle's HT_zeta(X - Lprev_oracle) at the same
    entries (arrays of equal shape: X, the other S^(k), the other and the oracle's L^(k-1)).
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
    explained = diff & ~inband & (dist <= dL)
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
