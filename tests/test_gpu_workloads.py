"""The CUDA path against the FP64 oracle on the two full-size Tucker workloads (GPU only):

  * 800^3 FP32, Gaussian Tucker rank (5,5,5), 30% outliers uniform in +-10 mean|L*|, v = 3
    (|I_i| = 101, |J_i| = 201), zeta0 = max|X|, gamma = 0.7, tol 1e-5, seed 0: the benchmark's
    workload, in the launch configuration it times (FULL scope, FP32 fused dense pass, 16-CTA
    refinement clusters), RTCUR-F and RTCUR-R (Sec. 3.4);
  * 100^3, Tucker rank (3,3,3), 20% outliers uniform in +-10 mean|L*|, v = 2 (|I_i| = 28,
    |J_i| = 56), same solver settings, RTCUR-F and RTCUR-R, both scopes.

The oracle runs Algorithm 1 in the SAMPLED scope: the iterates depend only on the sampled entries
(Sec. 3.3), so its (R, C_i, U_i^+) sequence is the FULL scope's too (pinned on the CPU). At 800^3
the GPU's whole L and S (2 GB each) are compared where the oracle can evaluate its Tucker state
entry by entry without forming the tensor:
  * every sampled entry of the last iteration (the subtensor R and the n fiber sets),
  * a seeded random 100 x 100 x 100 grid of entries (1e6),
  * four seeded whole mode-1 slabs (4 x 640,000 entries).
Checks: the iteration count, zeta^(k) to 1e-15 relative, e^(k) to 1e-4 relative (5e-8 absolute,
the FP32 floor of E = (X - S) - L), L to 1e-5 relative Frobenius over those entries, and the
support of S^(k) = HT_{zeta_k}(X - L^(k-1)) on the grid and the slabs: differences are split into
in-band (within 1e-6 zeta of the threshold), L-explained (|L_gpu - L_oracle| at L^(k-1) reaches
the distance to zeta) and unexplained, which must be 0. The counts are printed at the end of the
session."""
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


@pytest.fixture(scope="module")
def big():
    """The 800^3 problem, generated once for both variants."""
    return synth.make_tucker_problem((800, 800, 800), (5, 5, 5), 0.3, 3.0, seed=0, keep_truth=False,
                                     max_iter=100)


def _gpu_solve(X, p, idx, variant, max_iter, scope, want_S=True):
    """One solve through the C ABI with device outputs (kept on the device)."""
    import torch
    L = torch.empty_like(X)
    S = torch.empty_like(X) if want_S else None
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter,
                           rt.VARIANT_R if variant == "R" else rt.VARIANT_F, rt.make_options(scope=scope))
    try:
        res = rt.rtcur_solve(plan, X.data_ptr(), idx, L.data_ptr(), S.data_ptr() if want_S else 0,
                             torch.cuda.current_stream().cuda_stream, max_iter=max_iter)
    finally:
        rt.rtcur_destroy(plan)
    return res, L, S


def _take(T, coords):
    """Entries of a device tensor at integer coordinate arrays (one per mode, equal shapes)."""
    import torch
    idx = tuple(torch.from_numpy(np.ascontiguousarray(c.reshape(-1))).to(T.device) for c in coords)
    return T[idx].cpu().numpy().astype(np.float64).reshape(coords[0].shape)


def compare_with_oracle(p, sets, variant, X, res, L, S, Lprev, ref, rng_seed=1234, n_grid=100, n_slabs=4):
    """Entry-wise comparison of a GPU solve (device L, S and L^(k-1)) with the oracle's Tucker
    state: returns (relative Frobenius error of L over the compared entries, merged flip counts)."""
    dims = p.dims
    st, prev = ref["state"], ref["prev_state"]
    k = ref["iters"]
    last = sets[0] if variant == "F" else sets[k - 1]
    I, J = last["I"], last["J"]
    L_or, L_gpu = [], []
    # sampled entries of the last iteration: the subtensor and the fibers
    grid = np.meshgrid(*I, indexing="ij")
    L_or.append(st.eval_subtensor(I).ravel())
    L_gpu.append(_take(L, grid).ravel())
    for i in range(len(dims)):
        fc = O.fiber_coords(dims, i, J[i])
        L_or.append(st.eval_fibers(dims, i, J[i]).ravel())
        L_gpu.append(_take(L, [np.asarray(c) for c in fc]).ravel())
    # a seeded random grid and whole mode-1 slabs: L^(k) and the support of S^(k)
    rng = np.random.default_rng(rng_seed)
    groups = [[np.sort(rng.choice(d, size=min(d, n_grid), replace=False)) for d in dims]]
    for s in np.sort(rng.choice(dims[0], size=n_slabs, replace=False)):
        groups.append([np.array([s])] + [np.arange(d) for d in dims[1:]])
    flips = []
    for G in groups:
        coords = np.meshgrid(*G, indexing="ij")
        Xg = p.X[np.ix_(*G)].astype(np.float64)
        L_or.append(O.tucker_eval_subtensor(st.core, st.factors, G).ravel())
        L_gpu.append(_take(L, coords).ravel())
        Lp_or = prev.eval_subtensor(G)
        flips.append(CMP.support_flips(Xg, _take(S, coords), _take(Lprev, coords), Lp_or, ref["zeta"]))
    rel = CMP.rel_fro(np.concatenate(L_gpu), np.concatenate(L_or))
    return rel, CMP.merge_flips(flips)


@pytest.mark.parametrize("variant", ["F", "R"])
def test_800cubed_full_scope_matches_oracle(big, variant, parity_log):
    import torch
    p = big
    max_iter = 100
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=0, n_sets=max_iter if variant == "R" else 1)
    assert p.m == [101] * 3 and p.q == [201] * 3
    idx = synth.pack_index_sets(sets)
    X = torch.from_numpy(p.X).to("cuda:0")
    res, L, S = _gpu_solve(X, p, idx, variant, max_iter, rt.SCOPE_FULL)
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, max_iter, variant)
    assert res.status == rt.OK and ref["e"] <= p.tol
    assert res.iters == ref["iters"]
    np.testing.assert_allclose(res.zeta_hist, ref["hist"]["zeta"], rtol=1e-15)
    np.testing.assert_allclose(res.e_hist, ref["hist"]["e"], rtol=1e-4, atol=5e-8)
    # L^(k-1): the same solve one iteration shorter (the GPU's solves are deterministic)
    _, Lprev, _ = _gpu_solve(X, p, idx, variant, res.iters - 1, rt.SCOPE_FULL, want_S=False)
    rel, fl = compare_with_oracle(p, sets, variant, X, res, L, S, Lprev, ref)
    nnz_diff = int(np.max(np.abs(res.nnz_hist - np.asarray(ref["hist"]["nnz_sample"]))))
    parity_log(iters=res.iters, rel_L=f"{rel:.2e}", sampled_nnz_max_diff=nnz_diff, **fl)
    assert rel <= 1e-5
    assert fl["unexplained"] == 0, fl


@pytest.mark.parametrize("variant", ["F", "R"])
@pytest.mark.parametrize("scope", [rt.SCOPE_SAMPLED, rt.SCOPE_FULL])
def test_100cubed_matches_oracle(variant, scope, parity_log):
    """The 100^3 workload, whole tensors compared (the oracle forms L and S in full)."""
    import torch
    p = synth.make_tucker_problem((100, 100, 100), (3, 3, 3), 0.2, 2.0, seed=0, max_iter=100)
    assert p.m == [28] * 3 and p.q == [56] * 3
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=0, n_sets=100 if variant == "R" else 1)
    idx = synth.pack_index_sets(sets)
    X = torch.from_numpy(p.X).to("cuda:0")
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, 100, variant, keep_full=True)
    res, L, S = _gpu_solve(X, p, idx, variant, 100, scope)
    assert res.iters == ref["iters"]
    np.testing.assert_allclose(res.zeta_hist, ref["hist"]["zeta"], rtol=1e-15)
    # e^(k) moves with L on the unmasked sampled entries (E = X - L there): |de| <= ||dL|| / ||X||
    # on the sample. With the small samples of v = 2 (28 and 56) the late iterates carry ~2e-7
    # relative FP32 error in L, so the absolute allowance is 2e-7 here (5e-8 at 800^3).
    np.testing.assert_allclose(res.e_hist, ref["hist"]["e"], rtol=1e-4, atol=2e-7)
    Lh = L.cpu().numpy().astype(np.float64)
    rel = CMP.rel_fro(Lh, ref["L"])
    _, Lprev, _ = _gpu_solve(X, p, idx, variant, res.iters - 1, scope, want_S=False)
    fl = CMP.support_flips(p.X, S.cpu().numpy(), Lprev.cpu().numpy(), ref["prev_state"].full(p.dims), ref["zeta"])
    parity_log(iters=res.iters, rel_L=f"{rel:.2e}", **fl)
    assert rel <= 1e-5
    assert fl["unexplained"] == 0, fl
    # recovery of the planted low-rank part (Sec. 4.1 success criterion)
    assert CMP.rel_fro(Lh, p.L_star) <= 1e-3
