"""CUDA path vs the FP64 oracle, element by element, on seeded inputs (GPU only).

Tolerances (spec contract for the FP32 path): L within relative Frobenius 1e-5 of the
oracle; the support of S identical except entries with ||X - L| - zeta| <= 1e-6 zeta, which are
counted; the iteration count equal; e^(k) within 1e-4 relative or 5e-8 absolute. The absolute
part comes from the arithmetic: near convergence E = (X - S) - L is a difference of O(|X|)
FP32 values, so e carries an absolute error of a few FP32 ulps of |L| / |X| (measured ~2e-9)."""
import numpy as np
import pytest

from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

from gpu_helpers import rel_fro, run_gpu, support_mismatch

pytestmark = pytest.mark.gpu

CASES = [
    # dims (ragged, several Jacobi/tile sizes), ranks, alpha, upsilon, seed
    ((48, 40, 36), (3, 3, 3), 0.1, 3, 1),
    ((37, 45, 29), (2, 3, 2), 0.15, 3, 2),       # odd last mode: scalar dense path
    ((64, 30, 52), (4, 2, 3), 0.1, 4, 3),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("variant", ["F", "R"])
@pytest.mark.parametrize("scope", [rt.SCOPE_SAMPLED, rt.SCOPE_FULL])
def test_solve_matches_oracle(case, variant, scope):
    dims, ranks, alpha, ups, seed = case
    p = synth.make_tucker_problem(dims, ranks, alpha, ups, seed=seed, max_iter=60)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=seed, n_sets=60)
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, 60, variant, keep_full=True)
    res, L, S = run_gpu(p, sets, variant, scope=scope, max_iter=60)
    assert res.iters == ref["iters"]
    np.testing.assert_allclose(res.zeta_hist, ref["hist"]["zeta"], rtol=1e-15)
    np.testing.assert_allclose(res.e_hist, ref["hist"]["e"], rtol=1e-4, atol=5e-8)
    assert rel_fro(L, ref["L"]) <= 1e-5
    inband, outband = support_mismatch(S, ref, p.X)
    assert outband == 0, (inband, outband)
    if variant == "F" and res.iters > 12:
        assert res.warm_hits > 0  # the certified warm-started path engaged late in the solve


@pytest.mark.parametrize("variant", ["F", "R"])
def test_jacobi_eigensolver_path_matches_oracle(variant):
    dims, ranks, alpha, ups, seed = CASES[0]
    p = synth.make_tucker_problem(dims, ranks, alpha, ups, seed=seed, max_iter=60)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=seed, n_sets=60)
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, 60, variant, keep_full=True)
    res, L, S = run_gpu(p, sets, variant, max_iter=60, eig_method=rt.EIG_JACOBI)
    assert res.iters == ref["iters"]
    assert rel_fro(L, ref["L"]) <= 1e-5
