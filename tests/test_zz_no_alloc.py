"""The allocation-free dense threshold pass (for callers that cannot allocate device memory,
such as a process whose memory belongs to a fixed-budget pool) against the plan-based
rtcur_threshold_dense, on two calls in a row (GPU only). Collected last on purpose."""
import numpy as np
import pytest

from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_threshold_pass_twice():
    import torch
    import __graft_entry__ as ge
    ge.build()
    p = synth.make_tucker_problem((64, 48, 40), (3, 2, 3), 0.15, 3, seed=7)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=7)
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    X = torch.from_numpy(p.X).to(dev)
    S_ref = torch.empty_like(X)
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, 50, rt.VARIANT_F,
                           rt.make_options(scope=rt.SCOPE_FULL))
    try:
        rt.rtcur_begin(plan, X.data_ptr(), synth.pack_index_sets(sets), S_ref.data_ptr(), stream)
        rt.rtcur_iterate(plan, 4, stream)
        G, Bs, k, zeta_k = rt.rtcur_get_factors(plan, p.dims, p.ranks, stream)
        rt.rtcur_threshold_dense(plan, 1, stream)
        res = rt.rtcur_finish(plan, 0, 0, stream, max_iter=50)
    finally:
        rt.rtcur_destroy(plan)
    torch.cuda.synchronize()
    assert k == 4
    S_ref_h = S_ref.cpu().numpy()
    Gd = torch.from_numpy(np.ascontiguousarray(G.ravel())).to(dev)
    Bd = torch.from_numpy(np.concatenate([b.ravel() for b in Bs])).to(dev)
    zeta = p.gamma * zeta_k          # the plan's pass thresholds at zeta^(k+1) = gamma zeta^(k)
    outs = [torch.full_like(X, float("nan")) for _ in range(2)]
    torch.cuda.synchronize()
    for call in range(2):
        S = outs[call]
        free_before = torch.cuda.mem_get_info()[0]
        counts = rt.rtcur_threshold_dense_noalloc(p.dims, p.ranks, Gd.data_ptr(), Bd.data_ptr(),
                                                  X.data_ptr(), zeta, S.data_ptr(), stream)
        torch.cuda.synchronize()
        if call == 1:
            # the first call may load the library's kernels and look up the scratch array's address;
            # after it, a call takes no device memory at all
            assert torch.cuda.mem_get_info()[0] == free_before
        S_h = S.cpu().numpy()
        # same kernels on the same FP32 inputs: identical outputs (within any test tolerance)
        np.testing.assert_array_equal(S_h, S_ref_h)
        assert counts[1] == int(np.count_nonzero(S_ref_h)) == res.nnz_full
        assert abs(counts[0] - res.resid_full) <= 1e-12 * max(1.0, abs(res.resid_full))
