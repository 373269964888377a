"""Seeded synthetic inputs for RTCUR (robust tensor CUR), shared by the CUDA path and the oracle.

This module only draws random data and index sets. It holds none of the method's arithmetic:
no thresholding, no CUR, no pseudoinverse. Everything is host-side numpy with
``numpy.random.default_rng(seed)`` (PCG64), which gives the same stream on x86 and Arm.

Recipes (paper Sec. 4.1, "Synthetic Examples"):
  * low-rank part  L* = Y x_1 Y_1 x_2 ... x_n Y_n, core and factors i.i.d. N(0, 1);
  * sparse part    S*: exactly floor(alpha * N) positions drawn uniformly without replacement,
    values uniform in [-c * mean|L*|, c * mean|L*|] (c = 1 in the paper, c = 10 in the 800^3 and
    100^3 workloads used here);
  * sample sizes   |I_i| = ceil(v r_i ln d_i), |J_i| = ceil(v r_i ln prod_{j != i} d_j) (Sec. 4,
    sampling constant v), clamped to [r_i, d_i] and [r_i, prod_{j != i} d_j];
  * index sets     uniform without replacement, sorted ascending, 0-based (Algorithm 1, the
    sampling step). J_i indexes the columns of the mode-i unfolding X_(i) in row-major order
    of the remaining modes (last mode fastest).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "sample_sizes", "draw_index_set", "draw_index_sets", "draw_chidori_set", "draw_chidori_sets",
    "pack_index_sets",
    "tucker_lowrank", "planted_outliers", "make_tucker_problem", "make_video_problem",
    "make_batched_problems", "Problem",
]


def sample_sizes(dims, ranks, upsilon):
    """Return (m, q): m_i = |I_i|, q_i = |J_i| from the sampling-constant rule (Sec. 4)."""
    dims = [int(d) for d in dims]
    n = len(dims)
    m, q = [], []
    for i in range(n):
        other = 1
        for j in range(n):
            if j != i:
                other *= dims[j]
        r = int(ranks[i])
        mi = math.ceil(upsilon * r * math.log(dims[i])) if dims[i] > 1 else 1
        qi = math.ceil(upsilon * r * math.log(other)) if other > 1 else 1
        m.append(int(min(dims[i], max(r, mi))))
        q.append(int(min(other, max(r, qi))))
    return m, q


def draw_index_set(dims, m, q, rng):
    """One draw of {I_i}, {J_i}: uniform without replacement, sorted, int64."""
    n = len(dims)
    I, J = [], []
    for i in range(n):
        other = 1
        for j in range(n):
            if j != i:
                other *= int(dims[j])
        I.append(np.sort(rng.choice(int(dims[i]), size=int(m[i]), replace=False)).astype(np.int64))
        J.append(np.sort(rng.choice(other, size=int(q[i]), replace=False)).astype(np.int64))
    return {"I": I, "J": J}


def draw_chidori_set(dims, m, rng):
    """One draw for the Chidori form of the tensor CUR (the other named form of Sec. 2.2, defined in
    Cai, Hamm, Huang, Needell, "Mode-wise tensor decompositions"): I_i uniform as above, and J_i
    every column of X_(i) whose other-mode indices all lie in their I_j, i.e. the fibers through
    the core subtensor R = X(I_1, ..., I_n). Then |J_i| = prod_{j != i} m_j and C_i(I_i, :) is the
    mode-i unfolding of R. Column indices follow the same order (row-major over the remaining
    modes, last fastest), so J_i comes out sorted."""
    n = len(dims)
    I = [np.sort(rng.choice(int(dims[i]), size=int(m[i]), replace=False)).astype(np.int64) for i in range(n)]
    J = []
    for i in range(n):
        col = np.zeros(1, dtype=np.int64)
        for j in range(n):
            if j != i:
                col = (col[:, None] * int(dims[j]) + I[j][None, :]).reshape(-1)
        J.append(col)
    return {"I": I, "J": J}


def draw_chidori_sets(dims, m, seed, n_sets=1):
    """``n_sets`` independent Chidori draws from one seeded stream (see ``draw_chidori_set``)."""
    rng = np.random.default_rng([int(seed), 0xC41D])
    return [draw_chidori_set(dims, m, rng) for _ in range(n_sets)]


def draw_index_sets(dims, m, q, seed, n_sets=1):
    """``n_sets`` independent draws (1 for the fixed-index variant, one per iteration for the
    resampling variant), from one seeded stream."""
    rng = np.random.default_rng([int(seed), 0x5EED])
    return [draw_index_set(dims, m, q, rng) for _ in range(n_sets)]


def pack_index_sets(sets):
    """Flatten sets to the C-ABI layout: per set I_1..I_n then J_1..J_n, int64, contiguous."""
    parts = []
    for s in sets:
        parts.extend(s["I"])
        parts.extend(s["J"])
    return np.ascontiguousarray(np.concatenate(parts).astype(np.int64))


def tucker_lowrank(dims, ranks, rng, dtype=np.float64):
    """L* = Y x_i Y_i with Gaussian core and factors (Sec. 4.1). Built mode by mode with
    ``numpy.tensordot`` (a library contraction); returns (L*, core, factors)."""
    n = len(dims)
    core = rng.standard_normal(tuple(int(r) for r in ranks))
    factors = [rng.standard_normal((int(dims[i]), int(ranks[i]))) for i in range(n)]
    T = core
    for i in range(n):
        # contract axis i of T with the columns of factor i, put the new axis back at i
        T = np.moveaxis(np.tensordot(factors[i], T, axes=([1], [i])), 0, i)
    return np.ascontiguousarray(T.astype(dtype, copy=False)), core, factors


def _exact_size_support(N, k, rng):
    """Uniform k-subset of range(N) as a boolean mask. Small N: direct choice. Large N: a
    Bernoulli(k/N) mask, then uniformly random additions/removals until it holds exactly k
    (exchangeability keeps the subset uniform)."""
    mask = np.zeros(N, dtype=bool)
    if k <= 0:
        return mask
    if N <= (1 << 24):
        mask[rng.choice(N, size=k, replace=False)] = True
        return mask
    chunk = 1 << 24
    p = k / N
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        mask[s:e] = rng.random(e - s, dtype=np.float32) < p
    cnt = int(mask.sum())
    while cnt != k:
        need = k - cnt
        cand = rng.integers(0, N, size=abs(need) * 2 + 16)
        if need > 0:
            cand = np.unique(cand[~mask[cand]])
            cand = cand[rng.permutation(cand.size)][:need]
            mask[cand] = True
        else:
            cand = np.unique(cand[mask[cand]])
            cand = cand[rng.permutation(cand.size)][:-need]
            mask[cand] = False
        cnt = int(mask.sum())
    return mask


def planted_outliers(shape, alpha, scale, rng, dtype=np.float32):
    """S*: floor(alpha*N) uniform positions, values uniform in [-scale, scale] (Sec. 4.1)."""
    N = int(np.prod(shape))
    k = int(math.floor(alpha * N))
    mask = _exact_size_support(N, k, rng)
    S = np.zeros(N, dtype=dtype)
    idx = np.flatnonzero(mask)
    S[idx] = (rng.random(idx.size) * 2.0 - 1.0).astype(dtype) * dtype(scale)
    return S.reshape(shape)


@dataclass
class Problem:
    """One synthetic RTCUR problem and the solver settings it is meant to run with."""
    X: np.ndarray
    dims: tuple
    ranks: tuple
    m: list
    q: list
    zeta0: float
    gamma: float = 0.7
    tol: float = 1e-5
    max_iter: int = 100
    L_star: np.ndarray | None = None
    S_star: np.ndarray | None = None
    meta: dict = field(default_factory=dict)


def make_tucker_problem(dims, ranks, alpha, upsilon, seed=0, outlier_scale=10.0,
                        dtype=np.float32, zeta0=None, gamma=0.7, tol=1e-5, max_iter=100,
                        keep_truth=True):
    """X = L* + S* with a Gaussian Tucker L* and planted uniform outliers (Sec. 4.1).

    ``outlier_scale`` is the multiple of mean|L*| bounding the outlier values (1 in the paper,
    10 in the 100^3 / 800^3 workloads). ``zeta0=None`` means max|X|."""
    rng = np.random.default_rng(int(seed))
    dims = tuple(int(d) for d in dims)
    ranks = tuple(int(r) for r in ranks)
    L, _, _ = tucker_lowrank(dims, ranks, rng, dtype=np.float64 if np.prod(dims) <= (1 << 26) else np.float32)
    mean_abs = float(np.mean(np.abs(L), dtype=np.float64))
    S = planted_outliers(dims, alpha, outlier_scale * mean_abs, rng, dtype=np.float64 if L.dtype == np.float64 else np.float32)
    X = (L + S).astype(dtype)
    m, q = sample_sizes(dims, ranks, upsilon)
    z0 = float(np.max(np.abs(X))) if zeta0 is None else float(zeta0)
    return Problem(X=X, dims=dims, ranks=ranks, m=m, q=q, zeta0=z0, gamma=gamma, tol=tol,
                   max_iter=max_iter, L_star=L if keep_truth else None,
                   S_star=S if keep_truth else None,
                   meta={"seed": seed, "alpha": alpha, "upsilon": upsilon,
                         "outlier_scale": outlier_scale, "mean_abs_L": mean_abs})


def _dct_columns(d, k):
    """First k DCT-II basis columns cos(pi (2x+1) j / (2d)), j = 0..k-1 (column 0 is constant)."""
    x = np.arange(d, dtype=np.float64)[:, None]
    j = np.arange(k, dtype=np.float64)[None, :]
    return np.cos(np.pi * (2 * x + 1) * j / (2 * d))


def make_video_problem(H=240, W=320, colours=3, frames=600, ranks=(10, 10, 2, 4), upsilon=2,
                       seed=0, n_rects=40, gamma=0.7, tol=1e-5, max_iter=100):
    """Colour-video-shaped H x W x colour x frames tensor in [0, 1] (stand-in for the paper's
    video data of Sec. 4.2, which is not available here). Background: Tucker of rank ``ranks``
    with smooth cosine factors, each holding a constant column, affinely mapped into [0, 1].
    Foreground: ``n_rects`` axis-aligned rectangles of 20-60 px moving linearly, overwriting
    voxels with uniform [0, 1] values until a seed-chosen 5-10% of voxels are covered."""
    rng = np.random.default_rng(int(seed))
    dims = (H, W, colours, frames)
    facs = [_dct_columns(H, ranks[0]), _dct_columns(W, ranks[1]),
            _dct_columns(colours, ranks[2]), _dct_columns(frames, ranks[3])]
    core = rng.standard_normal(tuple(ranks)) / (1.0 + np.add.outer(
        np.add.outer(np.arange(ranks[0]), np.arange(ranks[1])),
        np.add.outer(np.arange(ranks[2]), np.arange(ranks[3]))))
    T = core
    for i in range(4):
        T = np.moveaxis(np.tensordot(facs[i], T, axes=([1], [i])), 0, i)
    lo, hi = float(T.min()), float(T.max())
    L = ((T - lo) / (hi - lo)).astype(np.float32)  # affine map keeps the multilinear rank
    X = L.copy()
    target = rng.uniform(0.05, 0.10)
    covered = np.zeros((H, W, frames), dtype=bool)
    rects = []
    for _ in range(n_rects):
        h, w = rng.integers(20, 61, size=2)
        y0, x0 = rng.uniform(0, H - h), rng.uniform(0, W - w)
        vy, vx = rng.uniform(-1.5, 1.5, size=2)
        t0 = int(rng.integers(0, frames))
        t1 = int(min(frames, t0 + rng.integers(frames // 8, frames // 2)))
        rects.append((int(h), int(w), y0, x0, vy, vx, t0, t1))
    for (h, w, y0, x0, vy, vx, t0, t1) in rects:
        for t in range(t0, t1):
            y = int(np.clip(y0 + vy * (t - t0), 0, H - h))
            x = int(np.clip(x0 + vx * (t - t0), 0, W - w))
            covered[y:y + h, x:x + w, t] = True
        if covered.mean() >= target:
            break
    ys, xs, ts = np.nonzero(covered)
    vals = rng.random((ys.size, colours)).astype(np.float32)
    for c in range(colours):
        X[ys, xs, c, ts] = vals[:, c]
    m, q = sample_sizes(dims, ranks, upsilon)
    return Problem(X=X, dims=dims, ranks=tuple(ranks), m=m, q=q, zeta0=1.0, gamma=gamma,
                   tol=tol, max_iter=max_iter, L_star=L, S_star=X - L,
                   meta={"seed": seed, "foreground_fraction": float(covered.mean()),
                         "upsilon": upsilon})


def make_batched_problems(count=64, dmin=64, dmax=320, rmin=2, rmax=10, amin=0.1, amax=0.4,
                          upsilon=3, seed0=0, outlier_scale=10.0):
    """``count`` independent 3-mode problems with uneven dims and ranks; problem b uses seed
    ``seed0 + b`` for its shape draw and its data."""
    out = []
    for b in range(count):
        rng = np.random.default_rng([int(seed0 + b), 0xBA7C])
        dims = tuple(int(x) for x in rng.integers(dmin, dmax + 1, size=3))
        ranks = tuple(int(x) for x in rng.integers(rmin, rmax + 1, size=3))
        alpha = float(rng.uniform(amin, amax))
        out.append(make_tucker_problem(dims, ranks, alpha, upsilon, seed=seed0 + b,
                                       outlier_scale=outlier_scale))
    return out
