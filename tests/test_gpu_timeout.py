"""Failure detection of the dense threshold pass (GPU only), without a GPU fault: every wait of
the pass on its shared-memory barriers is bounded. With the bound set to a single non-blocking
poll (rtcur_set_wait_limit) the first wait of the launch gives up before its copy has landed; the
pass then waits, with its default bound, for its own copies still in flight, records
RTCUR_ETIMEOUT and returns. The solve must stop and report RTCUR_ETIMEOUT, the context must stay
usable, and the next solve on the same plan, with the default bound restored, must give the same
result as before the timeout."""
import numpy as np
import pytest

from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

pytestmark = pytest.mark.gpu


def test_dense_pass_wait_timeout_is_reported_and_recoverable():
    import torch
    import __graft_entry__ as ge
    ge.build()
    p = synth.make_tucker_problem((64, 48, 40), (3, 2, 3), 0.15, 3, seed=9, max_iter=40)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=9)
    idx = synth.pack_index_sets(sets)
    X = torch.from_numpy(p.X).to("cuda:0")
    L0, S0 = torch.empty_like(X), torch.empty_like(X)
    L1, S1 = torch.empty_like(X), torch.empty_like(X)
    s = torch.cuda.current_stream().cuda_stream
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, 40, rt.VARIANT_F,
                           rt.make_options(scope=rt.SCOPE_FULL))
    try:
        ref = rt.rtcur_solve(plan, X.data_ptr(), idx, L0.data_ptr(), S0.data_ptr(), s, max_iter=40)
        assert ref.status == rt.OK and ref.iters > 1
        rt.rtcur_set_wait_limit(plan, 1, s)
        with pytest.raises(rt.RTCURError) as ei:
            rt.rtcur_solve(plan, X.data_ptr(), idx, L1.data_ptr(), S1.data_ptr(), s, max_iter=40)
        assert ei.value.status == rt.ETIMEOUT
        torch.cuda.synchronize()  # the context is still usable
        rt.rtcur_set_wait_limit(plan, 0, s)
        res = rt.rtcur_solve(plan, X.data_ptr(), idx, L1.data_ptr(), S1.data_ptr(), s, max_iter=40)
    finally:
        rt.rtcur_destroy(plan)
    assert res.status == rt.OK and res.iters == ref.iters
    np.testing.assert_array_equal(res.e_hist, ref.e_hist)
    assert torch.equal(L1, L0) and torch.equal(S1, S0)
