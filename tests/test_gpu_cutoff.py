"""The truncation SVD_r of Sec. 3.1 at its degenerate ends, against the FP64 oracle (GPU only).

SVD_r keeps the top r singular triplets of W_i = C_i(I_i, :) but drops those at or below the cutoff
max(|I_i|, |J_i|) 2^-24 s_1: the data are FP32, so smaller singular values are below their
resolution (the oracle's reading, pinned on the CPU). Two outlier-free problems reach the pinv's
exact path (singular vectors of the refined subspace, then the cutoff) instead of its
well-conditioned fast finish:
  * rank-deficient: a Tucker L* of multilinear rank (2,2,2) solved with ranks (3,3,3). Once the
    iterate is clean, sigma_3(W_i) is FP32 rounding noise, far below the cutoff; both sides keep 2
    singular values per mode and the library raises RTCUR_FLAG_RANK_DEFICIENT;
  * near-separated: rank (3,3,3) with the third column of every factor scaled by 1e-3, so
    sigma_3 / sigma_1 ~ 2e-4: below the fast finish's conditioning bound (sigma_r / sigma_1 > 1e-3),
    well above the cutoff (~4e-6 sigma_1 here); all 3 are kept and the flag stays clear. Its zeta0 = 2 max|X| makes the
    first threshold remove nothing (the closed-form special case: L^(1) = CUR(X), one iteration),
    so W_i is the FP32 data itself, sigma_4 sits at its rounding level and the gap stays clean.
    (From zeta0 = max|X| the first threshold removes the largest entries of X, W_i becomes full rank
    with sigma_4 near sigma_3, and that iterate's SVD_r is a near tie: parity unpinned there.)
Checks: the iteration count, zeta^(k) and e^(k) histories, L (relative Frobenius 1e-5), the kept
rank per mode (the trace of the projector C_i(I_i, :) U_i^+ from the exported pieces, against the
oracle's count), and the flag."""
import numpy as np
import pytest

from oracle import compare as CMP
from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


def _problem(dims, planted, solve_ranks, scale3, seed, upsilon=3.0, zeta_scale=1.0):
    """Outlier-free X = L* (FP32) with Gaussian core and factors; factor columns >= 2 scaled;
    zeta0 = zeta_scale max|X|."""
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(tuple(planted))
    factors = [rng.standard_normal((d, r)) for d, r in zip(dims, planted)]
    for F in factors:
        F[:, 2:] *= scale3
    L = O.tucker_full(core, factors)
    X = np.ascontiguousarray(L.astype(np.float32))
    m, q = synth.sample_sizes(dims, solve_ranks, upsilon)
    return synth.Problem(X=X, dims=tuple(dims), ranks=tuple(solve_ranks), m=m, q=q,
                         zeta0=zeta_scale * float(np.max(np.abs(X))), max_iter=80, L_star=L)


CASES = [
    # name, dims, planted ranks, solved ranks, scale of factor columns >= 2, variant, seed, zeta0 / max|X|
    ("rank_deficient_F", (60, 52, 44), (2, 2, 2), (3, 3, 3), 1.0, "F", 41, 1.0),
    ("rank_deficient_R", (48, 56, 40), (2, 2, 2), (3, 3, 3), 1.0, "R", 42, 1.0),
    ("rank_deficient_first_iterate", (60, 52, 44), (2, 2, 2), (3, 3, 3), 1.0, "F", 44, 2.0),
    ("near_separated_F", (60, 52, 44), (3, 3, 3), (3, 3, 3), 1e-3, "F", 43, 2.0),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_svd_r_cutoff_matches_oracle(case, parity_log):
    import torch
    name, dims, planted, ranks, scale3, variant, seed, zscale = case
    p = _problem(dims, planted, ranks, scale3, seed, zeta_scale=zscale)
    max_iter = p.max_iter
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=seed, n_sets=max_iter if variant == "R" else 1)
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, max_iter, variant, keep_full=True)
    X = torch.from_numpy(p.X).to("cuda:0")
    L = torch.empty_like(X)
    s = torch.cuda.current_stream().cuda_stream
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter,
                           rt.VARIANT_R if variant == "R" else rt.VARIANT_F, rt.make_options())
    try:
        res = rt.rtcur_solve(plan, X.data_ptr(), synth.pack_index_sets(sets), L.data_ptr(), 0, s,
                             max_iter=max_iter)
        R, Cs, Us, k = rt.rtcur_get_cur(plan, p.dims, p.m, p.q, s)
    finally:
        rt.rtcur_destroy(plan)
    assert res.iters == ref["iters"]
    np.testing.assert_allclose(res.zeta_hist, ref["hist"]["zeta"], rtol=1e-15)
    np.testing.assert_allclose(res.e_hist, ref["hist"]["e"], rtol=1e-4, atol=2e-7)
    rel = CMP.rel_fro(L.cpu().numpy(), ref["L"])
    last = sets[0] if variant == "F" else sets[k - 1]
    kept_gpu = [int(round(np.trace(Cs[i][last["I"][i]].astype(np.float64) @ Us[i]))) for i in range(3)]
    info = ref["info"]
    kept_or = [O.svd_truncated(info["C"][i][last["I"][i]], ranks[i])[1].size for i in range(3)]
    parity_log(case=name, iters=res.iters, rel_L=f"{rel:.2e}", kept_gpu=kept_gpu, kept_oracle=kept_or,
               flags=res.flags)
    assert rel <= 1e-5
    assert kept_gpu == kept_or
    if planted[0] < ranks[0]:
        assert kept_or == list(planted)
        assert res.flags & rt.FLAG_RANK_DEFICIENT
    else:
        assert kept_or == list(ranks)
        assert not (res.flags & rt.FLAG_RANK_DEFICIENT)
    assert CMP.rel_fro(L.cpu().numpy(), p.L_star) <= 1e-5  # outlier-free: L* is recovered
