"""Precision forms on the 4-mode colour-video-shaped workload (GPU only): a 240 x 320 x 3 x 600
FP32 tensor in [0, 1] (smooth Tucker background of rank (10, 10, 2, 4) plus moving rectangles,
the stand-in for the paper's colour videos), RTCUR-F with v = 2, FULL scope, each dense-pass
form (FP32 fused, BF16 split and TF32 on the tensor cores) against the FP64 oracle after 15
iterations.

Every form gives the oracle's iteration count, e^(k) history and L within relative Frobenius
1e-5 (the dense pass does not feed the sampled iterate). For S^(15) = HT_zeta(X - L^(14)) over the
whole tensor:
  * FP32 form: S equals, bit for bit, the host's FP32 evaluation of HT_zeta(X - L_gpu^(14)) with
    L_gpu^(14) materialised by the library (the dense pass and the materialisation evaluate L in
    the same FP32 order), and against the oracle every support difference lies where
    ||X - L^(14)| - zeta| is within 1e-6 zeta or within |L_gpu^(14) - L_oracle^(14)| at that entry:
    a flip caused by the FP32 evaluation of L, not by the thresholding (here zeta^(15) ~ 5e-3 while
    |L| ~ 0.5, so 1e-6 zeta alone is below FP32's resolution of L);
  * BF16 / TF32 forms: the same, with the form's evaluation error added (~2^-16 of max |L| for the
    BF16 split, ~2^-11 for TF32, times a safety factor)."""
import numpy as np
import pytest

from oracle import compare as CMP
from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

from gpu_helpers import rel_fro, run_gpu

pytestmark = pytest.mark.gpu

MAXIT = 15
BAND = {rt.FORM_FP32: 0.0, rt.FORM_BF16: 1e-4, rt.FORM_TF32: 4e-3}


@pytest.fixture(scope="module")
def video():
    import __graft_entry__ as ge
    ge.build()
    p = synth.make_video_problem(seed=0, upsilon=2, max_iter=MAXIT)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=0)
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, MAXIT, "F", keep_full=True)
    Lprev_or = ref["prev_state"].full(p.dims)                       # L_oracle^(14)
    dist = np.abs(np.abs(p.X.astype(np.float64) - Lprev_or) - ref["zeta"])
    # L_gpu^(14): the same deterministic trajectory stopped one iteration earlier
    _, Lprev_gpu, _ = run_gpu(p, sets, "F", scope=rt.SCOPE_FULL, max_iter=MAXIT - 1, want_S=False)
    return p, sets, ref, dist, np.abs(Lprev_gpu - Lprev_or), Lprev_gpu.astype(np.float32)


@pytest.mark.parametrize("form", [rt.FORM_FP32, rt.FORM_BF16, rt.FORM_TF32])
def test_video_form_matches_oracle(video, form, parity_log):
    p, sets, ref, dist, dL, Lprev32 = video
    res, L, S = run_gpu(p, sets, "F", scope=rt.SCOPE_FULL, max_iter=MAXIT, dense_form=form)
    assert res.iters == ref["iters"] == MAXIT
    np.testing.assert_allclose(res.e_hist[:MAXIT], ref["hist"]["e"], rtol=1e-4, atol=5e-8)
    assert rel_fro(L, ref["L"]) <= 1e-5
    if form == rt.FORM_FP32:
        D32 = p.X - Lprev32                                          # FP32, as on the GPU
        S_host = np.where(np.abs(D32) > np.float32(ref["zeta"]), D32, np.float32(0))
        np.testing.assert_array_equal(S.astype(np.float32), S_host)
    # support differences: in band / L-explained (the FP32 L^(k-1) difference plus the form's
    # evaluation bound) / unexplained, counted and logged
    fl = CMP.support_flips(p.X, S, Lprev32, ref["prev_state"].full(p.dims), ref["zeta"],
                           extra=BAND[form] * np.max(np.abs(ref["L"])))
    parity_log(form=form, iters=res.iters, rel_L=f"{rel_fro(L, ref['L']):.2e}", **fl)
    assert fl["unexplained"] == 0, fl
    assert res.nnz_full == int(np.count_nonzero(S))
