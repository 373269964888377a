"""Export of Algorithm 1's output, the Fiber CUR pieces (R, C_i, U_i^+) of Eq. (L=CUR) and
Eq. (R, C_i, U_i) (GPU only): L^(k) rebuilt on the host in FP64 as R x_i (C_i U_i^+) from the
exported pieces must match the library's own L^(k) (relative Frobenius 1e-5, the FP32 path's
tolerance), and each piece must match the oracle's (the cases recover their planted L*, so the
iterates are well conditioned): R and C_i (the sampled X - S^(k); they differ
from the oracle's only where S is nonzero, by the FP32 error of L there), U_i^+ through the
projector C_i(I_i, :) U_i^+, and A_i = C_i U_i^+ (1e-5)."""
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


CASES = [
    ((48, 40, 36), (3, 3, 3), 0.1, 3.0, "F", 5),
    ((37, 45, 29), (2, 3, 2), 0.15, 3.0, "R", 6),
    ((30, 24, 20, 16), (2, 2, 2, 2), 0.1, 4.0, "F", 7),
]


@pytest.mark.parametrize("case", CASES)
def test_exported_cur_pieces_rebuild_L_and_match_the_oracle(case):
    import torch
    dims, ranks, alpha, ups, variant, seed = case
    max_iter = 60
    p = synth.make_tucker_problem(dims, ranks, alpha, ups, seed=seed, max_iter=max_iter)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=seed, n_sets=max_iter if variant == "R" else 1)
    X = torch.from_numpy(p.X).to("cuda:0")
    L = torch.empty_like(X)
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter,
                           rt.VARIANT_R if variant == "R" else rt.VARIANT_F, rt.make_options())
    s = torch.cuda.current_stream().cuda_stream
    try:
        res = rt.rtcur_solve(plan, X.data_ptr(), synth.pack_index_sets(sets), L.data_ptr(), 0, s,
                             max_iter=max_iter)
        R, Cs, Us, k = rt.rtcur_get_cur(plan, p.dims, p.m, p.q, s)
    finally:
        rt.rtcur_destroy(plan)
    assert k == res.iters > 0
    Lg = L.cpu().numpy().astype(np.float64)
    A = [Ci.astype(np.float64) @ Ui for Ci, Ui in zip(Cs, Us)]
    L_rebuilt = O.tucker_full(R.astype(np.float64), A)
    assert CMP.rel_fro(L_rebuilt, Lg) <= 1e-5
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, max_iter, variant)
    assert ref["iters"] == k
    info = ref["info"]
    last = sets[0] if variant == "F" else sets[k - 1]
    assert CMP.rel_fro(R, info["R"]) <= 1e-5
    for i in range(len(dims)):
        assert CMP.rel_fro(Cs[i], info["C"][i]) <= 1e-5
        assert CMP.rel_fro(A[i], info["A"][i]) <= 1e-5
        # C_i(I_i, :) U_i^+ is the rank-r_i orthogonal projector Q_r Q_r^T (Sec. 3.1)
        Pm = Cs[i][last["I"][i]].astype(np.float64) @ Us[i]
        assert np.allclose(Pm, Pm.T, atol=1e-5) and abs(np.trace(Pm) - ranks[i]) <= 1e-4
    assert CMP.rel_fro(L_rebuilt, ref["state"].full(p.dims)) <= 1e-5
    assert CMP.rel_fro(L_rebuilt, p.L_star) <= 1e-3  # a well-posed case: the planted L* is recovered


def test_cur_export_before_any_iteration_is_rejected():
    import torch
    p = synth.make_tucker_problem((30, 28, 26), (2, 2, 2), 0.1, 3.0, seed=8, max_iter=10)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=8)
    X = torch.from_numpy(p.X).to("cuda:0")
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, 10, rt.VARIANT_F,
                           rt.make_options())
    s = torch.cuda.current_stream().cuda_stream
    try:
        rt.rtcur_begin(plan, X.data_ptr(), synth.pack_index_sets(sets), 0, s)
        with pytest.raises(rt.RTCURError) as ei:
            rt.rtcur_get_cur(plan, p.dims, p.m, p.q, s)
        assert ei.value.status == rt.EINVAL
    finally:
        rt.rtcur_destroy(plan)
