"""Plain, slow, FP64 CPU oracle for RTCUR (Robust Tensor CUR; Cai, Chao, Huang, Needell).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference leg may import or run this module. The CUDA library never calls it,
and it imports nothing from the CUDA side (it shares only the seeded input generators).

Every function follows one passage of the paper:
  * unfolding X_(k)                      -- Sec. 2.1, Definition "Tensor Matricization/Unfolding"
  * mode-k product X x_k A               -- Sec. 2.1, Definition "Mode-k Product"
  * Fiber CUR  A = R x_i (C_i U_i^+)     -- Sec. 2.2, Theorem (Fiber CUR characterization)
  * hard thresholding HT_zeta            -- Sec. 3.2, Eq. (HT) and the S update
  * partial (sampled) S update           -- Sec. 3.3, Eq. (partial S update)
  * L update with SVD_r                  -- Sec. 3.1, Eq. (L=CUR) and Eq. (R, C_i, U_i)
  * zeta decay zeta^{k+1} = gamma zeta^k -- Sec. 3.2
  * stopping error e^(k)                 -- Sec. 3.3, Eq. (rel_err)
  * RTCUR-F / RTCUR-R                    -- Sec. 3.4, Algorithm 1

Readings where the paper is silent:
  * indices are 0-based; J_i indexes columns of X_(i) in row-major order of the remaining
    modes (last mode fastest); sets are sorted (order does not change L);
  * zeta decays before the first thresholding (Algorithm 1 order), so S^(1) = HT_{gamma zeta0}(X);
  * HT keeps |x| > zeta strictly;
  * e^(0) = 1 (L^(0) = S^(0) = 0 gives E = X); a zero denominator gives e = 0;
  * SVD_r keeps the top r singular triplets except those with s_j <= max(m, q) * 2^-24 * s_1
    (the input tensor is FP32, so smaller singular values are below its resolution);
  * the residual written (X - S) at a thresholded entry equals L^(k) there.

The L state is kept as a Tucker-form pair (core, factors) with L = core x_i factors_i. After a
CUR update that pair is (R, A_i = C_i U_i^+) exactly as Eq. (L=CUR) writes it; any other
Tucker pair (for example one exported from another implementation) can be evaluated the same
way, which is what the one-step parity check uses.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "FP32_EPS", "unfold", "fold", "mode_product", "tucker_full", "hard_threshold",
    "other_mode_coords", "fiber_coords", "gather_subtensor", "gather_fibers",
    "tucker_eval_subtensor", "tucker_eval_fibers", "svd_truncated", "truncated_pinv",
    "fiber_cur", "relative_error", "rtcur_step", "rtcur", "RTCURState",
]

FP32_EPS = 2.0 ** -24  # unit roundoff of the FP32 input data (cutoff of SVD_r)


# --------------------------------------------------------------------------- Sec. 2.1
def unfold(X, k):
    """Mode-k unfolding X_(k) (d_k x prod_{j != k} d_j). Column order: row-major over the
    remaining modes, last mode fastest (the paper leaves the order open)."""
    return np.moveaxis(np.asarray(X), k, 0).reshape(X.shape[k], -1)


def fold(M, k, shape):
    """Inverse of ``unfold`` for a tensor of the given shape."""
    shape = tuple(shape)
    rest = shape[:k] + shape[k + 1:]
    return np.moveaxis(M.reshape((shape[k],) + rest), 0, k)


def mode_product(X, A, k):
    """Y = X x_k A, defined by Y_(k) = A X_(k) (Definition "Mode-k Product")."""
    shape = list(X.shape)
    Yk = np.asarray(A, dtype=np.float64) @ unfold(X, k)
    shape[k] = A.shape[0]
    return fold(Yk, k, shape)


def tucker_full(core, factors):
    """core x_1 F_1 x_2 ... x_n F_n (Definition "Tucker decomposition")."""
    T = np.asarray(core, dtype=np.float64)
    for k, F in enumerate(factors):
        T = mode_product(T, F, k)
    return T


# --------------------------------------------------------------------------- Sec. 3.2
def hard_threshold(D, zeta):
    """HT_zeta: keep an entry when |x| > zeta, zero otherwise (strict inequality)."""
    D = np.asarray(D, dtype=np.float64)
    return np.where(np.abs(D) > zeta, D, 0.0)


# ------------------------------------------------------------- sampled positions (Sec. 3.3)
def other_mode_coords(dims, i, J):
    """Decode column indices J of X_(i) into the coordinates of the other modes.
    Returns a list of n arrays; entry i is None."""
    dims = [int(d) for d in dims]
    J = np.asarray(J, dtype=np.int64)
    coords = [None] * len(dims)
    rem = J.copy()
    for l in reversed(range(len(dims))):
        if l == i:
            continue
        coords[l] = rem % dims[l]
        rem = rem // dims[l]
    return coords


def fiber_coords(dims, i, J):
    """Full coordinates of the fibers C_i = X_(i)(:, J): n arrays of shape (d_i, |J|)."""
    dims = [int(d) for d in dims]
    oc = other_mode_coords(dims, i, J)
    out = []
    for l in range(len(dims)):
        if l == i:
            out.append(np.broadcast_to(np.arange(dims[i])[:, None], (dims[i], len(J))))
        else:
            out.append(np.broadcast_to(oc[l][None, :], (dims[i], len(J))))
    return out


def gather_subtensor(X, I):
    """X(I_1, ..., I_n) (notation of Sec. 1.2)."""
    return np.asarray(X, dtype=np.float64)[np.ix_(*I)]


def gather_fibers(X, i, J):
    """X_(i)(:, J_i): d_i x |J_i|."""
    return np.asarray(X, dtype=np.float64)[tuple(fiber_coords(X.shape, i, J))]


def tucker_eval_subtensor(core, factors, I):
    """L(I_1..I_n) for L = core x_i F_i, as core x_i F_i(I_i, :) (no full tensor formed; the
    point made at the end of Sec. 3.1)."""
    return tucker_full(core, [F[np.asarray(Ii)] for F, Ii in zip(factors, I)])


def tucker_eval_fibers(core, factors, dims, i, J):
    """L_(i)(:, J) for L = core x_l F_l: each fiber j with other coordinates p_l is
    F_i (core x_{l != i} F_l(p_l, :)) -- the staged evaluation of Sec. 3.3."""
    n = len(dims)
    oc = other_mode_coords(dims, i, J)
    Z = np.asarray(core, dtype=np.float64)           # axes: the n core modes
    Z = np.broadcast_to(Z, (len(J),) + Z.shape)      # batch axis 0 over the fibers
    # contract every mode l != i with the row F_l(p_l(b), :) of its own fiber b
    axes_left = list(range(n))                       # core mode -> current axis (minus batch)
    for l in reversed(range(n)):
        if l == i:
            continue
        rows = np.asarray(factors[l], dtype=np.float64)[oc[l]]     # (nb, r_l)
        ax = 1 + axes_left.index(l)
        Z = np.moveaxis(Z, ax, -1)                   # (nb, ..., r_l)
        Z = np.einsum("b...c,bc->b...", Z, rows)
        axes_left.remove(l)
    # Z is (nb, r_i): apply F_i
    return np.asarray(factors[i], dtype=np.float64) @ Z.T     # (d_i, nb)


# --------------------------------------------------------------------------- Sec. 3.1
def svd_truncated(W, r, eps=FP32_EPS):
    """SVD_r(W): the top r singular triplets of W (numpy LAPACK SVD as the library step),
    dropping singular values s_j <= max(m, q) * eps * s_1. Returns (Q_r, s_r, V_r)."""
    W = np.asarray(W, dtype=np.float64)
    U, s, Vt = np.linalg.svd(W, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return U[:, :0], s[:0], Vt[:0].T
    tau = max(W.shape) * eps * s[0]
    k = int(min(r, np.count_nonzero(s > tau)))
    return U[:, :k], s[:k], Vt[:k].T


def truncated_pinv(W, r, eps=FP32_EPS):
    """(SVD_r(W))^+ = V_r diag(1/s_r) Q_r^T (Moore-Penrose pseudoinverse of the rank-r part)."""
    Q, s, V = svd_truncated(W, r, eps)
    return (V / s[None, :]) @ Q.T


def fiber_cur(R, C, I, ranks, eps=FP32_EPS):
    """Fiber CUR factors A_i = C_i (SVD_{r_i}(C_i(I_i, :)))^+ (Eq. (L=CUR) / Eq. (R, C_i, U_i)).
    L = R x_i A_i is then the Fiber CUR approximation of the Theorem in Sec. 2.2."""
    A = []
    for i, Ci in enumerate(C):
        W = Ci[np.asarray(I[i]), :]
        A.append(Ci @ truncated_pinv(W, ranks[i], eps))
    return A


# --------------------------------------------------------------------------- Sec. 3.3
def relative_error(ER, EC, XR, XC):
    """e^(k) of Eq. (rel_err): sum of Frobenius norms (not squared) over the subtensor and the
    n fiber sets, divided by the same sum for X. A zero denominator gives 0."""
    num = np.linalg.norm(ER) + sum(np.linalg.norm(E) for E in EC)
    den = np.linalg.norm(XR) + sum(np.linalg.norm(Xc) for Xc in XC)
    return 0.0 if den == 0.0 else float(num / den)


class RTCURState:
    """L^(k) in Tucker form (core, factors); L^(0) = 0 is ``core=None``."""

    def __init__(self, core=None, factors=None):
        self.core = core
        self.factors = factors

    def eval_subtensor(self, I):
        if self.core is None:
            return np.zeros(tuple(len(x) for x in I))
        return tucker_eval_subtensor(self.core, self.factors, I)

    def eval_fibers(self, dims, i, J):
        if self.core is None:
            return np.zeros((int(dims[i]), len(J)))
        return tucker_eval_fibers(self.core, self.factors, dims, i, J)

    def full(self, dims):
        if self.core is None:
            return np.zeros(tuple(int(d) for d in dims))
        return tucker_full(self.core, self.factors)


def rtcur_step(X, state, sets, zeta, ranks, eps=FP32_EPS):
    """One pass of Algorithm 1's loop body at threshold ``zeta`` (already decayed):
    Step (I), the sampled S update of Eq. (partial S update), and Step (II), the Fiber CUR
    L update of Eq. (L=CUR), then e^(k+1) of Eq. (rel_err) on the same sets.

    Returns (new_state, info) with the sampled pieces (R, C_i, U_i^+ factors, the S masks)."""
    X = np.asarray(X)
    dims = X.shape
    n = X.ndim
    I, J = sets["I"], sets["J"]
    # Step (I): S^(k+1) = HT(X - L^(k)) only on the subtensor and the fibers
    XR = gather_subtensor(X, I)
    SR = hard_threshold(XR - state.eval_subtensor(I), zeta)
    XC = [gather_fibers(X, i, J[i]) for i in range(n)]
    SC = [hard_threshold(XC[i] - state.eval_fibers(dims, i, J[i]), zeta) for i in range(n)]
    # Step (II): R = (X - S)(I_1..I_n), C_i = (X - S)_(i)(:, J_i), A_i = C_i U_i^+
    R = XR - SR
    C = [XC[i] - SC[i] for i in range(n)]
    A = fiber_cur(R, C, I, ranks, eps)
    new = RTCURState(R, A)
    # e^(k+1) with E = X - L^(k+1) - S^(k+1) on the sets of this iteration
    ER = R - new.eval_subtensor(I)
    EC = [C[i] - new.eval_fibers(dims, i, J[i]) for i in range(n)]
    e = relative_error(ER, EC, XR, XC)
    info = {"R": R, "C": C, "A": A, "SR": SR, "SC": SC, "XR": XR, "XC": XC, "e": e,
            "nnz_sample": int(np.count_nonzero(SR) + sum(np.count_nonzero(s) for s in SC))}
    return new, info


def rtcur(X, ranks, index_sets, zeta0, gamma, tol, max_iter, variant="F", scope="sampled",
          eps=FP32_EPS, keep_full=False, inband_rel=1e-6):
    """Algorithm 1 (RTCUR). ``variant`` "F" uses index_sets[0] throughout, "R" uses
    index_sets[k] at iteration k (Sec. 3.4). ``scope`` "full" additionally forms the whole
    S^(k+1) = HT(X - L^(k)) each iteration (the literal Step (I)); the iterates do not depend
    on it. Returns a dict with the iteration count, histories, the final Fiber CUR pieces
    (R, C_i, A_i = C_i U_i^+), and optionally the full L and S."""
    X = np.asarray(X)
    dims = X.shape
    Xd = X.astype(np.float64)
    state = RTCURState()
    prev = state
    zeta = float(zeta0)
    k = 0
    e = 1.0
    hist = {"e": [], "zeta": [], "nnz_sample": [], "nnz_full": [], "resid_full": [], "inband_full": []}
    info = None
    S_full = None
    while e > tol and k < max_iter:
        sets = index_sets[0] if variant == "F" else index_sets[k]
        zeta = gamma * zeta
        if scope == "full":
            D = Xd - state.full(dims)
            S_full = hard_threshold(D, zeta)
            hist["nnz_full"].append(int(np.count_nonzero(S_full)))
            hist["resid_full"].append(float(np.sum((D - S_full) ** 2)))
            hist["inband_full"].append(int(np.count_nonzero(np.abs(np.abs(D) - zeta) <= inband_rel * zeta)))
        prev = state
        state, info = rtcur_step(Xd, state, sets, zeta, ranks, eps)
        k += 1
        e = info["e"]
        hist["e"].append(e)
        hist["zeta"].append(zeta)
        hist["nnz_sample"].append(info["nnz_sample"])
    out = {"iters": k, "e": e, "zeta": zeta, "hist": hist, "state": state, "prev_state": prev,
           "info": info}
    if keep_full:
        out["L"] = state.full(dims)
        if S_full is None:
            S_full = hard_threshold(Xd - prev.full(dims), zeta)
        out["S"] = S_full
    return out
