"""Dense-pass forms (FULL scope) on the GPU: FP32 fused, FP32 plain (literal chain, unfused),
BF16 (3-term split on tensor cores) and TF32 (tensor cores).

The CUR iterates read only sampled entries, so every form must give the same iteration count,
e^(k) history and L as the FP32 form. The whole-tensor S may differ only where |X - L| lies within
the form's evaluation error of zeta: the relative error of L is about 2^-24 r (FP32 plain and
fused orders differ), ~2^-16 for the BF16 split (the dropped lo*lo term) and ~2^-11 for TF32; the
bands below are those bounds times a safety factor, relative to max |L|."""
import numpy as np
import pytest

from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu

BAND = {rt.FORM_FP32_PLAIN: 2e-6, rt.FORM_BF16: 1e-4, rt.FORM_TF32: 4e-3}
# Fraction of entries whose support may differ. Near convergence zeta^(k) falls below the TF32
# evaluation error of L (~1e-3 max|L|), so the many near-zero residuals of non-outliers sit inside
# the TF32 band and may flip; the band containment above is the guarantee, the count a sanity cap.
MAXFRAC = {rt.FORM_FP32_PLAIN: 1e-3, rt.FORM_BF16: 1e-3, rt.FORM_TF32: 5e-2}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


SHAPES = [
    ((48, 40, 64), (3, 3, 4), 21),     # whole row tiles, one partial column block
    ((37, 45, 60), (2, 3, 5), 22),     # ragged last row tile, a partial TMA box
    ((20, 26, 260), (3, 2, 3), 23),    # three column blocks, the last one 4 columns wide
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("form", [rt.FORM_FP32_PLAIN, rt.FORM_BF16, rt.FORM_TF32])
def test_form_matches_fp32_form(form, shape):
    dims, ranks, seed = shape
    p = synth.make_tucker_problem(dims, ranks, 0.1, 3, seed=seed, max_iter=40)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=seed)
    ref, L0, S0 = run_gpu(p, sets, "F", scope=rt.SCOPE_FULL, max_iter=40)
    res, L1, S1 = run_gpu(p, sets, "F", scope=rt.SCOPE_FULL, max_iter=40, dense_form=form)
    assert res.iters == ref.iters
    np.testing.assert_array_equal(res.e_hist, ref.e_hist)
    np.testing.assert_array_equal(L1, L0)
    # S^(k) = HT_{zeta_k}(X - L^(k-1)): support differences only inside the form's band
    diff = (S1 != 0) != (S0 != 0)
    # where exactly one form kept an entry, its S value is X - L there: |X - L| is known
    absD = np.where(S0 != 0, np.abs(S0), np.abs(S1))
    zeta = ref.zeta
    band = BAND[form] * np.max(np.abs(L0))
    assert np.all(np.abs(absD[diff] - zeta) <= band + 1e-6 * zeta), int(diff.sum())
    assert diff.sum() <= MAXFRAC[form] * diff.size


@pytest.mark.parametrize("form", [rt.FORM_FP32_PLAIN, rt.FORM_BF16, rt.FORM_TF32])
def test_form_matches_oracle(form, parity_log):
    """Each form against the FP64 oracle itself (not only against the FP32 form): the same
    iterates, and S^(k)'s support differences in band / L-explained (the FP32 L^(k-1) difference
    plus the form's evaluation band) / unexplained, the last required to be 0."""
    from oracle import compare as CMP
    from oracle import rtcur_oracle as O
    from gpu_helpers import rel_fro
    dims, ranks, seed = SHAPES[0]
    p = synth.make_tucker_problem(dims, ranks, 0.1, 3, seed=seed, max_iter=40)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=seed)
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, 40, "F", keep_full=True)
    res, L, S = run_gpu(p, sets, "F", scope=rt.SCOPE_FULL, max_iter=40, dense_form=form)
    assert res.iters == ref["iters"]
    np.testing.assert_allclose(res.e_hist, ref["hist"]["e"], rtol=1e-4, atol=5e-8)
    rel = rel_fro(L, ref["L"])
    assert rel <= 1e-5
    _, Lprev, _ = run_gpu(p, sets, "F", scope=rt.SCOPE_FULL, max_iter=res.iters - 1, want_S=False,
                          dense_form=form)
    fl = CMP.support_flips(p.X, S, Lprev, ref["prev_state"].full(p.dims), ref["zeta"],
                           extra=BAND[form] * np.max(np.abs(ref["L"])))
    parity_log(form=form, iters=res.iters, rel_L=f"{rel:.2e}", **fl)
    assert fl["unexplained"] == 0, fl


def test_tensor_core_forms_reject_unsupported_shapes():
    # d_n % 4 != 0 (TMA row stride), d_n > 1024, BF16 with 3 r_n > 16, TF32 with r_n > 8
    for dims, ranks, form in (([20, 20, 30], [2, 2, 2], rt.FORM_BF16),
                              ([8, 8, 1028], [2, 2, 2], rt.FORM_TF32),
                              ([20, 20, 32], [2, 2, 6], rt.FORM_BF16),
                              ([20, 20, 32], [2, 2, 9], rt.FORM_TF32)):
        with pytest.raises(rt.RTCURError):
            rt.rtcur_create(dims, ranks, [8, 8, 16], [16, 16, 16], 1.0, 0.7, 1e-5, 5, 0,
                            rt.make_options(scope=rt.SCOPE_FULL, dense_form=form))
