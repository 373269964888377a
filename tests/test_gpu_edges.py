"""Edge and degenerate cases of the CUDA path against the FP64 oracle (GPU only): the matrix case
(n = 2) and a small 4-mode tensor, rank 1, no outliers, index sets covering a whole mode, a single
iteration, no iteration at all (tol >= 1: L^(0) = 0), |I_i| above the tridiagonal eigensolver's
limit (the Jacobi path), the largest rank, zeta0 = max|X| computed on the device, and a NaN on
the sample (RTCUR_ENONFINITE). Tolerances are those of the main parity tests, except that e^(k)
gets an absolute allowance of 2e-7: where a case recovers its L* exactly (no outliers, small
4-mode tensors) e falls to the FP32 floor of E = (X - S) - L, a few units of 2^-24 relative to |X|.
The ranks are admissible (each r_i at most the product of the others), so sigma_r / sigma_{r+1}
grows as the outliers are removed; with an inadmissible rank the truncation keeps noise
directions, the SVD_r is ill-conditioned and parity is unpinned there."""
import numpy as np
import pytest

from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

from gpu_helpers import flip_counts, rel_fro, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


def _check(p, sets, variant, max_iter, parity_log, scope=rt.SCOPE_SAMPLED, **opt):
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, max_iter, variant, keep_full=True)
    res, L, S = run_gpu(p, sets, variant, scope=scope, max_iter=max_iter, **opt)
    assert res.iters == ref["iters"]
    if ref["iters"]:
        np.testing.assert_allclose(res.e_hist[:res.iters], ref["hist"]["e"], rtol=1e-4, atol=2e-7)
        np.testing.assert_allclose(res.zeta_hist[:res.iters], ref["hist"]["zeta"], rtol=1e-15)
    rel = rel_fro(L, ref["L"])
    assert rel <= 1e-5 or np.linalg.norm(ref["L"]) == 0.0
    # Outside the 1e-6 zeta band a difference is allowed only where the FP32 evaluation of
    # L^(k-1) explains it (|L_gpu - L_oracle| at that entry reaches its distance to zeta), which
    # happens once zeta^(k) is far below |L|; every difference is counted and logged.
    fl = flip_counts(p, sets, variant, ref, S, scope=scope, max_iter=max_iter, **opt)
    parity_log(iters=res.iters, rel_L=f"{rel:.2e}", **fl)
    assert fl["unexplained"] == 0, fl
    return res, ref, L


CASES = [
    # name, dims, ranks, alpha, upsilon, variant, max_iter, extra make_tucker_problem args
    ("matrix", (120, 90), (3, 3), 0.1, 3.0, "F", 60, {}),
    ("matrix_R", (96, 140), (2, 2), 0.15, 3.0, "R", 60, {}),
    ("four_modes", (20, 18, 16, 14), (2, 2, 2, 2), 0.1, 3.0, "F", 60, {}),
    ("rank1", (40, 36, 44), (1, 1, 1), 0.1, 3.0, "F", 60, {}),
    ("no_outliers", (40, 36, 44), (2, 3, 2), 0.0, 3.0, "F", 60, {}),
    ("whole_mode", (12, 50, 60), (3, 2, 2), 0.1, 3.0, "F", 60, {}),   # m_0 clamps to d_0 = 12
    ("one_iteration", (40, 36, 44), (2, 2, 2), 0.2, 3.0, "F", 1, {}),
    ("jacobi_path", (200, 40, 60), (10, 4, 4), 0.1, 3.0, "F", 40, {}),  # m_0 = 159 > 128
    ("rank16", (96, 64, 48), (16, 8, 4), 0.05, 2.0, "F", 40, {}),
    ("zeta0_maxabs", (40, 36, 44), (2, 2, 2), 0.2, 3.0, "R", 60, {"zeta0": -1.0}),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_edge_case_matches_oracle(case, parity_log):
    name, dims, ranks, alpha, ups, variant, max_iter, kw = case
    p = synth.make_tucker_problem(dims, ranks, alpha, ups, seed=31, max_iter=max_iter, **kw)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=31, n_sets=max_iter if variant == "R" else 1)
    if name == "zeta0_maxabs":
        # zeta0 <= 0: the device computes max|X| (exact in FP32, so it equals the host's value)
        ref = O.rtcur(p.X, p.ranks, sets, float(np.max(np.abs(p.X))), p.gamma, p.tol, max_iter, variant,
                      keep_full=True)
        res, L, _ = run_gpu(p, sets, variant, max_iter=max_iter)
        assert res.iters == ref["iters"]
        np.testing.assert_allclose(res.zeta_hist[:res.iters], ref["hist"]["zeta"], rtol=1e-15)
        assert rel_fro(L, ref["L"]) <= 1e-5
        return
    if name == "whole_mode":
        assert p.m[0] == dims[0]
    if name == "jacobi_path":
        assert max(p.m) > 128
    _check(p, sets, variant, max_iter, parity_log)


def test_no_iteration_when_tol_is_at_least_one():
    p = synth.make_tucker_problem((30, 28, 26), (2, 2, 2), 0.1, 3.0, seed=32, tol=1.0, max_iter=10)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=32)
    res, L, S = run_gpu(p, sets, "F", scope=rt.SCOPE_FULL, max_iter=10)
    assert res.iters == 0 and res.e == 1.0 and res.status == rt.OK
    assert np.all(L == 0.0) and np.all(S == 0.0)  # L^(0) = 0; no threshold has run


def test_nan_on_the_sample_is_reported():
    p = synth.make_tucker_problem((30, 28, 26), (2, 2, 2), 0.1, 3.0, seed=33, max_iter=10)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=33)
    I = sets[0]["I"]
    p.X[I[0][0], I[1][0], I[2][0]] = np.nan  # an entry of the subtensor R
    with pytest.raises(rt.RTCURError) as ei:
        run_gpu(p, sets, "F", max_iter=10)
    assert ei.value.status == rt.ENONFINITE
