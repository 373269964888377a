"""The BF16 copy of X for the sampled step (options.sample_x = BF16), against the FP64 oracle
(GPU only).

With this option the sampled step (Step (I) on the sample, Eq. partial S update, and the gathers
of R and C_i, Sec. 3.3) reads X rounded to BF16 (round to nearest even), while the FULL scope's
dense pass keeps reading the FP32 X. Two comparisons per case:
  * parity: the oracle run on the same BF16-rounded tensor (the rounding done here, on the host,
    from the FP32 bits) gives the iterates the GPU must reproduce: iteration count, zeta/e
    histories, L, and the dense S = HT_zeta(X - L^(k-1)) over the FP32 X against the oracle's
    L^(k-1) with 0 unexplained support differences. The rounding puts every sampled value 2^-9
    off its low-rank-plus-sparse model, so late iterates fit noise: as zeta falls below that
    noise, S absorbs most entries and the trajectory becomes sensitive (as in the non-recovering
    100^3 solve). The bounds for e^(k) and L are therefore max(5e-8, 3 x) and max(1e-5, 3 x) the
    change that a relative 1e-7 perturbation of every L evaluation causes in the oracle's own
    solve of the rounded tensor (computed here);
  * the price: the same solve against the oracle on the FP32 tensor (the default path's
    reference). The BF16 rounding (up to 2^-9 relative per sampled value) moves L by about that
    much; the iteration count, L's relative error and the support differences are reported, and L
    must stay within 1e-2.
Cases: two small ragged shapes (F and R) and the 800^3 bench workload (F and R, FULL scope)."""
import numpy as np
import pytest

from oracle import compare as CMP
from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

from gpu_helpers import trajectory_sensitivity

pytestmark = pytest.mark.gpu


def bf16_round(X):
    """FP32 -> BF16 -> FP32, round to nearest even on the bit pattern (finite values)."""
    u = np.ascontiguousarray(X, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(X.shape)


def test_bf16_round_matches_torch():
    import torch
    x = np.random.default_rng(3).standard_normal(100000).astype(np.float32) * 1e3
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(bf16_round(x), ref)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


def _solve(p, sets, variant, scope, max_iter, want_prev):
    import torch
    X = torch.from_numpy(p.X).to("cuda:0")
    L, S = torch.empty_like(X), torch.empty_like(X)
    Lp = torch.empty_like(X) if want_prev else None
    s = torch.cuda.current_stream().cuda_stream
    idx = synth.pack_index_sets(sets)
    v = rt.VARIANT_R if variant == "R" else rt.VARIANT_F
    opt = rt.make_options(scope=scope, sample_x=rt.SAMPLE_X_BF16)
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter, v, opt)
    try:
        res = rt.rtcur_solve(plan, X.data_ptr(), idx, L.data_ptr(), S.data_ptr(), s, max_iter=max_iter)
    finally:
        rt.rtcur_destroy(plan)
    if want_prev and res.iters > 1:
        plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, res.iters - 1, v, opt)
        try:
            rt.rtcur_solve(plan, X.data_ptr(), idx, Lp.data_ptr(), 0, s, max_iter=res.iters - 1)
        finally:
            rt.rtcur_destroy(plan)
    elif want_prev:
        Lp.zero_()
    return res, L, S, Lp


def _take(T, coords):
    import torch
    idx = tuple(torch.from_numpy(np.ascontiguousarray(np.asarray(c).reshape(-1))).to(T.device) for c in coords)
    return T[idx].cpu().numpy().astype(np.float64).reshape(np.asarray(coords[0]).shape)


def _check(p, sets, variant, scope, max_iter, parity_log, full_tensors, monkeypatch):
    Xb = bf16_round(p.X)
    ref_b = O.rtcur(Xb, p.ranks, sets, p.zeta0, p.gamma, p.tol, max_iter, variant, keep_full=full_tensors)
    ref_f = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, max_iter, variant, keep_full=full_tensors)
    sens_L, sens_e = trajectory_sensitivity(monkeypatch, Xb, p, sets, variant, ref_b, max_iter)
    tol_L, tol_e = max(1e-5, 3.0 * sens_L), max(5e-8, 3.0 * sens_e)
    res, L, S, Lp = _solve(p, sets, variant, scope, max_iter, want_prev=True)
    assert res.iters == ref_b["iters"]
    np.testing.assert_allclose(res.zeta_hist, ref_b["hist"]["zeta"], rtol=1e-15)
    np.testing.assert_allclose(res.e_hist, ref_b["hist"]["e"], rtol=1e-4, atol=tol_e)
    out = {}
    for tag, ref in (("bf16_data", ref_b), ("fp32_data", ref_f)):
        if full_tensors:
            Lh = L.cpu().numpy().astype(np.float64)
            rel = CMP.rel_fro(Lh, ref["L"])
            fl = CMP.support_flips(p.X, S.cpu().numpy(), Lp.cpu().numpy(), ref["prev_state"].full(p.dims), ref["zeta"])
        else:
            k = ref["iters"]
            last = sets[0] if variant == "F" else sets[k - 1]
            groups = CMP.entry_groups(p.dims)
            orc = CMP.oracle_values(ref, p.dims, last, groups)
            grid = [np.meshgrid(*G, indexing="ij") for G in groups]
            if ref["iters"] == res.iters:
                L_sample = np.concatenate([_take(L, c).ravel() for c in CMP.sampled_coords(p.dims, last)])
            else:  # another iteration count: the last sets may differ (R); compare the grids only
                L_sample, orc = np.zeros(0), dict(orc, L_sample=np.zeros(0))
            rel, fl = CMP.compare_entries(p.X, groups, orc, L_sample, [_take(L, c) for c in grid],
                                          [_take(S, c) for c in grid], [_take(Lp, c) for c in grid], ref["zeta"])
        out[tag] = (ref["iters"], rel, fl)
    it_f, rel_f, fl_f = out["fp32_data"]
    parity_log(variant=variant, iters=res.iters, rel_L_vs_bf16_oracle=f"{out['bf16_data'][1]:.2e}",
               tol_L=f"{tol_L:.2e}", tol_e=f"{tol_e:.2e}",
               unexplained_vs_bf16_oracle=out["bf16_data"][2]["unexplained"],
               iters_fp32_oracle=it_f, rel_L_vs_fp32_oracle=f"{rel_f:.2e}",
               flips_vs_fp32_oracle=fl_f["flips"], L_explained_vs_fp32=fl_f["L_explained"])
    assert out["bf16_data"][1] <= tol_L
    assert out["bf16_data"][2]["unexplained"] == 0, out["bf16_data"][2]
    assert rel_f <= 1e-2


CASES = [((48, 40, 36), (3, 3, 3), 0.1, 3.0, "F", 1), ((37, 45, 29), (2, 3, 2), 0.15, 3.0, "R", 2)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("scope", [rt.SCOPE_SAMPLED, rt.SCOPE_FULL])
def test_bf16_sampled_copy_small(case, scope, parity_log, monkeypatch):
    dims, ranks, alpha, ups, variant, seed = case
    p = synth.make_tucker_problem(dims, ranks, alpha, ups, seed=seed, max_iter=60)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=seed, n_sets=60 if variant == "R" else 1)
    _check(p, sets, variant, scope, 60, parity_log, full_tensors=True, monkeypatch=monkeypatch)


@pytest.fixture(scope="module")
def big():
    return synth.make_tucker_problem((800, 800, 800), (5, 5, 5), 0.3, 3.0, seed=0, keep_truth=False,
                                     max_iter=100)


@pytest.mark.parametrize("variant", ["F", "R"])
def test_bf16_sampled_copy_800cubed(big, variant, parity_log, monkeypatch):
    sets = synth.draw_index_sets(big.dims, big.m, big.q, seed=0, n_sets=100 if variant == "R" else 1)
    _check(big, sets, variant, rt.SCOPE_FULL, 100, parity_log, full_tensors=False, monkeypatch=monkeypatch)
