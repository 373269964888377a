"""Batched form (rtcur_solve_batched): problems of uneven dims, ranks, sample sizes, variants and
scopes solved by one graph launch give exactly the results of solving each alone (the kernels
are deterministic and the batch shares no state between problems), and match the FP64 oracle
(GPU only)."""
import numpy as np
import pytest

from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth

from gpu_helpers import rel_fro

pytestmark = pytest.mark.gpu

SPECS = [
    # dims, ranks, alpha, upsilon, variant, scope, seed
    ((40, 52, 36), (2, 3, 2), 0.2, 3.0, "R", rt.SCOPE_SAMPLED, 10),
    ((64, 33, 47), (4, 2, 3), 0.1, 3.0, "F", rt.SCOPE_SAMPLED, 11),
    ((30, 30, 30), (2, 2, 2), 0.3, 3.0, "R", rt.SCOPE_SAMPLED, 12),
    ((72, 48, 40), (3, 3, 4), 0.15, 3.0, "F", rt.SCOPE_FULL, 13),
    ((45, 61, 38), (5, 2, 3), 0.25, 3.0, "R", rt.SCOPE_SAMPLED, 14),
]
MAXIT = 60


@pytest.fixture(scope="module")
def batch():
    import torch
    import __graft_entry__ as ge
    ge.build()
    probs = []
    for dims, ranks, alpha, ups, variant, scope, seed in SPECS:
        p = synth.make_tucker_problem(dims, ranks, alpha, ups, seed=seed, max_iter=MAXIT)
        sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=seed, n_sets=MAXIT if variant == "R" else 1)
        probs.append((p, sets, variant, scope))

    def plans():
        return [rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, MAXIT,
                                rt.VARIANT_R if v == "R" else rt.VARIANT_F, rt.make_options(scope=sc))
                for p, _, v, sc in probs]

    Xs = [torch.from_numpy(p.X).cuda() for p, _, _, _ in probs]
    Ls = [torch.empty_like(x) for x in Xs]
    Ss = [torch.empty_like(x) for x in Xs]
    idx = [synth.pack_index_sets(s) for _, s, _, _ in probs]
    stream = torch.cuda.current_stream().cuda_stream
    pl = plans()
    res_b = rt.rtcur_solve_batched(pl, [x.data_ptr() for x in Xs], idx, [l.data_ptr() for l in Ls],
                                   [s.data_ptr() for s in Ss], stream, max_iter=MAXIT)
    torch.cuda.synchronize()
    Lb = [l.cpu().numpy() for l in Ls]
    Sb = [s.cpu().numpy() for s in Ss]
    # a second call reuses the cached graph
    res_b2 = rt.rtcur_solve_batched(pl, [x.data_ptr() for x in Xs], idx, [l.data_ptr() for l in Ls],
                                    [s.data_ptr() for s in Ss], stream, max_iter=MAXIT)
    torch.cuda.synchronize()
    Lb2 = [l.cpu().numpy() for l in Ls]
    # each alone
    res_s, Ls1, Ss1 = [], [], []
    for i, pi in enumerate(pl):
        r = rt.rtcur_solve(pi, Xs[i].data_ptr(), idx[i], Ls[i].data_ptr(), Ss[i].data_ptr(), stream,
                           max_iter=MAXIT)
        torch.cuda.synchronize()
        res_s.append(r)
        Ls1.append(Ls[i].cpu().numpy())
        Ss1.append(Ss[i].cpu().numpy())
    # a different list (a sub-batch, reordered) rebuilds the graph
    sub = [pl[3], pl[0]]
    res_sub = rt.rtcur_solve_batched(sub, [Xs[3].data_ptr(), Xs[0].data_ptr()], [idx[3], idx[0]],
                                     [Ls[3].data_ptr(), Ls[0].data_ptr()], None, stream, max_iter=MAXIT)
    torch.cuda.synchronize()
    Lsub = [Ls[3].cpu().numpy(), Ls[0].cpu().numpy()]
    with pytest.raises(rt.RTCURError):
        rt.rtcur_solve_batched([pl[0], pl[0]], [Xs[0].data_ptr()] * 2, [idx[0]] * 2, None, None, stream)
    for x in pl:
        rt.rtcur_destroy(x)
    return dict(probs=probs, res_b=res_b, res_b2=res_b2, res_s=res_s, Lb=Lb, Lb2=Lb2, Sb=Sb, Ls1=Ls1,
                Ss1=Ss1, res_sub=res_sub, Lsub=Lsub)


def test_batched_equals_each_alone(batch):
    for i in range(len(SPECS)):
        a, b = batch["res_b"][i], batch["res_s"][i]
        assert a.iters == b.iters and a.e == b.e and a.zeta == b.zeta, i
        np.testing.assert_array_equal(batch["Lb"][i], batch["Ls1"][i])
        np.testing.assert_array_equal(batch["Sb"][i], batch["Ss1"][i])


def test_cached_graph_and_sub_batch(batch):
    for i in range(len(SPECS)):
        assert batch["res_b2"][i].iters == batch["res_b"][i].iters
        np.testing.assert_array_equal(batch["Lb2"][i], batch["Lb"][i])
    assert batch["res_sub"][0].iters == batch["res_s"][3].iters
    assert batch["res_sub"][1].iters == batch["res_s"][0].iters
    np.testing.assert_array_equal(batch["Lsub"][0], batch["Ls1"][3])
    np.testing.assert_array_equal(batch["Lsub"][1], batch["Ls1"][0])


def test_uneven_iteration_counts_all_converge(batch):
    its = [r.iters for r in batch["res_b"]]
    assert len(set(its)) > 1  # problems stop at different iterations inside the one launch
    for r in batch["res_b"]:
        assert r.status == rt.OK and r.e <= 1e-5


@pytest.mark.parametrize("i", [0, 3])
def test_batched_matches_oracle(batch, i):
    p, sets, variant, scope = batch["probs"][i]
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, MAXIT, variant, keep_full=True)
    assert batch["res_b"][i].iters == ref["iters"]
    assert rel_fro(batch["Lb"][i].astype(np.float64), ref["L"]) <= 1e-5


def test_autotuner_picks_a_converging_configuration(tmp_path):
    import torch
    from paper_2108_10448_gb300 import autotune
    probs = [synth.make_tucker_problem(d, r, 0.2, 3.0, seed=s)
             for d, r, s in (((40, 36, 44), (2, 3, 2), 20), ((52, 40, 30), (3, 2, 2), 21))]
    X = [torch.from_numpy(p.X).cuda() for p in probs]
    cache = str(tmp_path / "tune.json")
    out = autotune.tune_batch(X, [p.dims for p in probs], [p.ranks for p in probs],
                              [p.zeta0 for p in probs], variant="R", clusters=(4, 16),
                              upsilons=(3.0,), cache_path=cache)
    assert out["cluster"] in (4, 16) and out["upsilon"] == 3.0
    assert len(out["table"]) == 2 and all(r.get("converged") for r in out["table"])
    assert out["ms"] == min(r["ms"] for r in out["table"])
    again = autotune.tune_batch(X, [p.dims for p in probs], [p.ranks for p in probs],
                                [p.zeta0 for p in probs], variant="R", clusters=(4, 16),
                                upsilons=(3.0,), cache_path=cache)
    assert again == out  # served from the cache
