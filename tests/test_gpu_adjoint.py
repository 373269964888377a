"""The hand-written adjoint (rtcur_backward, behind a torch.autograd.Function) against the FP64
adjoint oracle and against central finite differences of the FP64 forward with frozen masks
(GPU only).

Workload: K = 10 unrolled RTCUR-F iterations on a 3-mode 200^3 FP32 tensor, Tucker rank
(5, 5, 5), 20% outliers, loss = ||L^(K) - L*||_F^2; the gradient with respect to X.

Tolerances. The forward runs in FP32 (sampled values, L evaluations) with an FP64 pinv; the
adjoint recomputes every pinv piece in FP64 from the recorded FP32 sampled values. The GPU and
oracle gradients are compared in relative Frobenius norm with the bound 1e-4 (the north-star
target for agreement with finite differences); the finite differences use the FP64 oracle
(h = 1e-3 along unit directions, masks checked unchanged), and their agreement is measured as
|fd - <g, v>| / ||g|| per direction and as the relative error of the 32-vector of directional
derivatives, both bounded by 1e-4."""
import numpy as np
import pytest

from oracle import rtcur_adjoint as AD
from paper_2108_10448_gb300 import synth

pytestmark = pytest.mark.gpu

K = 10


@pytest.fixture(scope="module")
def c5():
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2108_10448_gb300 import rtcur as rt
    from paper_2108_10448_gb300.autograd import rtcur_unrolled
    p = synth.make_tucker_problem((200, 200, 200), (5, 5, 5), 0.2, 3.0, seed=0, keep_truth=True)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=0)
    idx = synth.pack_index_sets(sets)
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, 0.0, K, rt.VARIANT_F,
                           rt.make_options(checkpoint=K))
    X = torch.from_numpy(p.X).cuda().requires_grad_(True)
    Lstar = torch.from_numpy(p.L_star.astype(np.float32)).cuda()
    L = rtcur_unrolled(X, plan, idx, K)
    loss = ((L.double() - Lstar.double()) ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    out = {"p": p, "sets": sets, "L": L.detach().cpu().numpy().astype(np.float64),
           "g": X.grad.cpu().numpy().astype(np.float64)}
    # same seed through the C ABI directly, to check the binding adds nothing
    s = torch.cuda.current_stream().cuda_stream

    def vjp(dL):
        dL = torch.as_tensor(dL).cuda().float().contiguous()
        dX = torch.empty_like(dL)
        rt.rtcur_backward(plan, dL.data_ptr(), dX.data_ptr(), s)
        torch.cuda.synchronize()
        return dL.cpu().numpy().astype(np.float64), dX.cpu().numpy().astype(np.float64)

    out["dL"], out["g_abi"] = vjp(2.0 * (L.detach().double() - Lstar.double()))
    # the oracle's frozen-mask forward; its adjoint on the same seed dL
    Lo, tape = AD.frozen_forward(p.X, p.ranks, sets, p.zeta0, p.gamma, K)
    out["Lo"], out["tape"] = Lo, tape
    out["go"] = AD.rtcur_vjp(p.X, tape, p.ranks, out["dL"])
    # the GPU adjoint applied to the oracle's residual: the gradient the FP64 differences see
    _, out["g_fd"] = vjp(2.0 * (Lo - p.L_star))
    rt.rtcur_destroy(plan)
    return out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_forward_matches_oracle(c5):
    assert _rel(c5["L"], c5["Lo"]) <= 1e-5


def test_autograd_equals_the_abi_call(c5):
    np.testing.assert_array_equal(c5["g"], c5["g_abi"])


def test_gradient_matches_oracle(c5):
    g, go = c5["g"], c5["go"]
    assert np.count_nonzero(go) > 0
    assert _rel(g, go) <= 1e-4, _rel(g, go)
    # zero off the sample, as in the oracle
    assert np.all(g[go == 0.0] == 0.0)


def test_gradient_matches_central_differences(c5):
    p, sets, tape = c5["p"], c5["sets"], c5["tape"]
    X = p.X.astype(np.float64)
    g = c5["g_fd"]
    base = [(t["mR"], t["mC"]) for t in tape]
    rng = np.random.default_rng(7)
    h = 1e-3
    fds, ans = [], []
    nd, tries = 0, 0
    while nd < 32 and tries < 64:
        tries += 1
        v = rng.standard_normal(X.shape)
        v /= np.linalg.norm(v)
        vals = []
        flipped = False
        for sgn in (1.0, -1.0):
            L, tp = AD.frozen_forward(X + sgn * h * v, p.ranks, sets, p.zeta0, p.gamma, K)
            for t, (mR, mC) in zip(tp, base):
                if not (np.array_equal(t["mR"], mR) and all(np.array_equal(a, b) for a, b in zip(t["mC"], mC))):
                    flipped = True
            vals.append(np.sum((L - p.L_star) ** 2))
        if flipped:  # a mask would flip: not a direction of the frozen-mask derivative
            continue
        fds.append((vals[0] - vals[1]) / (2 * h))
        ans.append(float(np.sum(g * v)))
        nd += 1
    assert nd == 32
    fds, ans = np.array(fds), np.array(ans)
    gn = np.linalg.norm(g)
    assert np.max(np.abs(fds - ans)) / gn <= 1e-4
    assert np.linalg.norm(fds - ans) / np.linalg.norm(fds) <= 1e-4
