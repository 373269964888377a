"""Plain FP64 CPU oracle for the adjoint (reverse-mode derivative) of K unrolled RTCUR iterations.

TEST INFRASTRUCTURE ONLY, like rtcur_oracle.py: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference leg may import or run it; the CUDA library never calls it.

What is differentiated. K iterations of Algorithm 1's loop body (Sec. 3.4) with the sampled
S update of Eq. (partial S update) and the Fiber CUR update of Eq. (L=CUR) give
L^(K) = R^(K) x_i A_i^(K), A_i = C_i U_i^+ with U_i^+ = (SVD_{r_i}(C_i(I_i,:)))^+. The map
X -> L^(K) is piecewise smooth: hard thresholding (Eq. (HT)) is differentiated almost everywhere,
i.e. with every support mask frozen at the value the forward pass took. With frozen masks each
sampled value entering R and C_i is

    V_p = L^(k)(p)   if the mask is set (|X_p - L^(k)(p)| > zeta^(k+1)),
    V_p = X_p        otherwise,

so X receives the adjoint of the unmasked slots and L^(k) (the previous iteration's factors)
that of the masked ones.

Readings:
  * the truncated pseudoinverse is differentiated where rank(U_i) >= r_i and sigma_{r_i} >
    sigma_{r_i + 1} (a.e.); the SVD_r cutoff is not active there;
  * U_i^+ = W^T Z with W = C_i(I_i,:), Z = sum_{j<=r} lambda_j^-1 u_j u_j^T over the top r
    eigenpairs of M = W W^T (the same matrix as V_r Sigma_r^-1 Q_r^T); Z is a spectral function of
    M and its derivative is the Daleckii-Krein divided-difference formula;
  * a sample position that occurs in several slots (R and fibers, or two fibers) contributes once
    per slot, as it enters the forward pass once per slot.
"""
from __future__ import annotations

import numpy as np

from .rtcur_oracle import (RTCURState, fiber_coords, fiber_cur, gather_fibers, gather_subtensor,
                           mode_product, other_mode_coords, truncated_pinv, unfold)

__all__ = ["frozen_forward", "tucker_vjp", "pinv_vjp", "rtcur_vjp", "fiber_z"]

_LETTERS = "abcdefgh"


def frozen_forward(X, ranks, index_sets, zeta0, gamma, K, variant="F", masks=None):
    """K iterations of Algorithm 1 (sampled scope). With ``masks=None`` the masks are computed
    (|X - L^(k)| > zeta^(k+1) on each slot); otherwise ``masks[k] = (mask_R, [mask_C_i])`` are
    used as given (frozen). Returns (L^(K) as a full tensor, tape); ``tape[k]`` holds iteration
    k+1's masks, R, C_i, A_i and index sets."""
    X = np.asarray(X, dtype=np.float64)
    dims = X.shape
    n = X.ndim
    state = RTCURState()
    zeta = float(zeta0)
    tape = []
    for k in range(K):
        sets = index_sets[0] if variant == "F" else index_sets[k]
        I, J = sets["I"], sets["J"]
        zeta = gamma * zeta
        XR = gather_subtensor(X, I)
        LR = state.eval_subtensor(I)
        XC = [gather_fibers(X, i, J[i]) for i in range(n)]
        LC = [state.eval_fibers(dims, i, J[i]) for i in range(n)]
        if masks is None:
            mR = np.abs(XR - LR) > zeta
            mC = [np.abs(XC[i] - LC[i]) > zeta for i in range(n)]
        else:
            mR, mC = masks[k]
        R = np.where(mR, LR, XR)
        C = [np.where(mC[i], LC[i], XC[i]) for i in range(n)]
        A = fiber_cur(R, C, I, ranks)
        tape.append({"mR": mR, "mC": mC, "R": R, "C": C, "A": A, "I": I, "J": J, "zeta": zeta})
        state = RTCURState(R, A)
    return state.full(dims), tape


def tucker_vjp(core, factors, Lbar):
    """Adjoint of L = core x_1 F_1 ... x_n F_n (Sec. 2.1 mode products):
    core_bar = Lbar x_i F_i^T (all i) and F_bar_i = Lbar_(i) (core x_{j != i} F_j)_(i)^T."""
    n = len(factors)
    cb = np.asarray(Lbar, dtype=np.float64)
    for i in range(n):
        cb = mode_product(cb, np.asarray(factors[i]).T, i)
    Fb = []
    for i in range(n):
        Y = np.asarray(core, dtype=np.float64)
        for j in range(n):
            if j != i:
                Y = mode_product(Y, factors[j], j)
        Fb.append(unfold(Lbar, i) @ unfold(Y, i).T)
    return cb, Fb


def pinv_vjp(W, r, Pbar):
    """Adjoint of P = (SVD_r(W))^+ at W (m x q, sigma_r > sigma_{r+1}, sigma_r > 0).

    P = W^T Z with Z = U_r diag(1/lambda_r) U_r^T, (lambda, U) the eigenpairs of M = W W^T in
    descending order. dP = dW^T Z + W^T dZ, and the Daleckii-Krein formula gives
    dZ = U (F o (U^T dM U)) U^T with F_jk = (f(l_j) - f(l_k)) / (l_j - l_k), F_jj = f'(l_j) for
    f = 1/l on the top r and 0 on the rest. With dM = dW W^T + W dW^T the adjoint is
    W_bar = Z Pbar^T + 2 Mbar W,  Mbar = U (F o (U^T sym(W Pbar) U)) U^T."""
    W = np.asarray(W, dtype=np.float64)
    Pbar = np.asarray(Pbar, dtype=np.float64)
    M = W @ W.T
    lam, U = np.linalg.eigh(M)
    lam, U = lam[::-1], U[:, ::-1]
    m = lam.size
    top = np.arange(m) < r
    F = np.zeros((m, m))
    for j in range(m):
        for k in range(m):
            if top[j] and top[k]:
                F[j, k] = -1.0 / (lam[j] * lam[k])
            elif top[j] and not top[k]:
                F[j, k] = 1.0 / (lam[j] * (lam[j] - lam[k]))
            elif top[k] and not top[j]:
                F[j, k] = 1.0 / (lam[k] * (lam[k] - lam[j]))
    Ur = U[:, :r]
    Z = (Ur / lam[:r][None, :]) @ Ur.T
    Zb = W @ Pbar
    Zb = 0.5 * (Zb + Zb.T)
    Mb = U @ (F * (U.T @ Zb @ U)) @ U.T
    return Z @ Pbar.T + 2.0 * Mb @ W


def fiber_z(R, A, dims, i, J):
    """z_j = R contracted on every mode l != i with the row A_l(p_l(j), :) of fiber j
    (m_i x |J|); the fiber values are then A_i z_j (the staged evaluation of Sec. 3.3)."""
    n = len(dims)
    oc = other_mode_coords(dims, i, J)
    core = _LETTERS[:n]
    ops = [np.asarray(R, dtype=np.float64)]
    subs = [core]
    for l in range(n):
        if l != i:
            ops.append(np.asarray(A[l], dtype=np.float64)[oc[l]])
            subs.append("z" + core[l])
    return np.einsum(",".join(subs) + "->" + core[i] + "z", *ops)


def _eval_vjp(R, A, dims, I, J, LbR, LbC):
    """Adjoint of the slot evaluations of L = R x_i A_i: the subtensor L(I_1..I_n) and the
    fibers L_(i)(:, J_i). Returns (R_bar, [A_bar_i])."""
    n = len(dims)
    A = [np.asarray(a, dtype=np.float64) for a in A]
    Ab = [np.zeros_like(a) for a in A]
    # subtensor: L_R = R x_i A_i(I_i, :)
    Rb, Fb = tucker_vjp(R, [A[i][np.asarray(I[i])] for i in range(n)], LbR)
    for i in range(n):
        Ab[i][np.asarray(I[i])] += Fb[i]
    core = _LETTERS[:n]
    for i in range(n):
        oc = other_mode_coords(dims, i, J[i])
        Z = fiber_z(R, A, dims, i, J[i])                 # m_i x q
        Ab[i] += LbC[i] @ Z.T
        Zb = A[i].T @ LbC[i]                              # m_i x q
        rows = {l: A[l][oc[l]] for l in range(n) if l != i}
        # R_bar += sum_j zbar_j (mode i) outer A_l(p_l(j), :) (modes l != i)
        ops = [Zb] + [rows[l] for l in range(n) if l != i]
        subs = [core[i] + "z"] + ["z" + core[l] for l in range(n) if l != i]
        Rb = Rb + np.einsum(",".join(subs) + "->" + core, *ops)
        # A_l(p_l(j), :) += R contracted with zbar_j and the other rows
        for l in range(n):
            if l == i:
                continue
            ops = [np.asarray(R, dtype=np.float64), Zb] + [rows[t] for t in range(n) if t not in (i, l)]
            subs = [core, core[i] + "z"] + ["z" + core[t] for t in range(n) if t not in (i, l)]
            G = np.einsum(",".join(subs) + "->z" + core[l], *ops)
            np.add.at(Ab[l], oc[l], G)
    return Rb, Ab


def rtcur_vjp(X, tape, ranks, dL):
    """d<dL, L^(K)>/dX for the frozen-mask forward pass recorded in ``tape`` (reverse sweep
    over the K iterations)."""
    X = np.asarray(X, dtype=np.float64)
    dims = X.shape
    n = X.ndim
    dX = np.zeros(dims)
    last = tape[-1]
    Rb, Ab = tucker_vjp(last["R"], last["A"], np.asarray(dL, dtype=np.float64))
    for k in reversed(range(len(tape))):
        t = tape[k]
        I, J = t["I"], t["J"]
        Cb = []
        for i in range(n):
            C = t["C"][i]
            Ii = np.asarray(I[i])
            W = C[Ii]
            P = truncated_pinv(W, ranks[i])
            cb = Ab[i] @ P.T                              # A_i = C_i P_i
            cb[Ii] += pinv_vjp(W, ranks[i], C.T @ Ab[i])  # through P_i = pinv_r(C_i(I_i, :))
            Cb.append(cb)
        # unmasked slots carry X, masked ones the previous L
        dX[np.ix_(*[np.asarray(x) for x in I])] += np.where(t["mR"], 0.0, Rb)
        for i in range(n):
            np.add.at(dX, tuple(fiber_coords(dims, i, J[i])), np.where(t["mC"][i], 0.0, Cb[i]))
        if k == 0:
            break
        LbR = np.where(t["mR"], Rb, 0.0)
        LbC = [np.where(t["mC"][i], Cb[i], 0.0) for i in range(n)]
        prev = tape[k - 1]
        Rb, Ab = _eval_vjp(prev["R"], prev["A"], dims, I, J, LbR, LbC)
    return dX
