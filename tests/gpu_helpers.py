"""Helpers shared by the GPU tests: run the CUDA path through the C ABI and the oracle on the
same seeded inputs."""
import numpy as np

from oracle import rtcur_oracle as O
from paper_2108_10448_gb300 import rtcur as rt
from paper_2108_10448_gb300 import synth


def run_gpu(p, sets, variant, scope=rt.SCOPE_SAMPLED, max_iter=None, want_L=True, want_S=True, **opt):
    import torch
    max_iter = max_iter or p.max_iter
    dev = torch.device("cuda:0")
    X = torch.from_numpy(np.ascontiguousarray(p.X)).to(dev)
    L = torch.empty_like(X) if want_L else None
    S = torch.empty_like(X) if want_S else None
    o = rt.make_options(scope=scope, **opt)
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter,
                           rt.VARIANT_R if variant == "R" else rt.VARIANT_F, o)
    try:
        res = rt.rtcur_solve(plan, X.data_ptr(), synth.pack_index_sets(sets),
                             L.data_ptr() if want_L else 0, S.data_ptr() if want_S else 0,
                             torch.cuda.current_stream().cuda_stream, max_iter=max_iter)
    finally:
        rt.rtcur_destroy(plan)
    return (res, L.cpu().numpy().astype(np.float64) if want_L else None,
            S.cpu().numpy().astype(np.float64) if want_S else None)


def rel_fro(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def flip_counts(p, sets, variant, ref, S, scope=None, extra=0.0, max_iter=None, **opt):
    """Support differences of a whole-tensor GPU S^(k) against the oracle's, as in-band /
    L-explained / unexplained counts (oracle.compare.support_flips). L_gpu^(k-1) comes from the
    same deterministic solve stopped one iteration earlier (only when there is a difference
    outside the band to explain). ``extra`` widens the L-explained test by a form's evaluation
    bound."""
    from oracle import compare as CMP
    Lor = ref["prev_state"].full(p.dims)
    fl = CMP.support_flips(p.X, S, Lor, Lor, ref["zeta"], extra=extra)
    if fl["flips"] > fl["inband"]:
        if ref["iters"] > 1:
            kw = dict(opt)
            if scope is not None:
                kw["scope"] = scope
            _, Lprev, _ = run_gpu(p, sets, variant, max_iter=ref["iters"] - 1, want_S=False, **kw)
        else:
            Lprev = np.zeros_like(Lor)
        fl = CMP.support_flips(p.X, S, Lprev, Lor, ref["zeta"], extra=extra)
    return fl


def support_mismatch(S_gpu, ref, X, band_rel=1e-6):
    """Support differences between the GPU's S^(k) and the oracle's, split into entries inside
    the band ||X - L^(k-1)| - zeta| <= band_rel * zeta (allowed) and outside it (not allowed)."""
    zeta = ref["zeta"]
    D = X.astype(np.float64) - ref["prev_state"].full(X.shape)
    band = np.abs(np.abs(D) - zeta) <= band_rel * zeta
    diff = (S_gpu != 0) != (ref["S"] != 0)
    return int(np.count_nonzero(diff & band)), int(np.count_nonzero(diff & ~band))


def trajectory_sensitivity(monkeypatch, X, p, sets, variant, ref, max_iter, rel=1e-7, seed=5):
    """How far the oracle's own solve moves when every evaluation of L^(k) on the sample is
    perturbed by a relative ``rel`` (seeded noise; 1e-7 is the size of an FP32 evaluation error):
    the conditioning of the whole trajectory, from the oracle alone. Returns (relative Frobenius
    change of the final L, largest absolute change of e^(k)); the solve ``ref`` is the unperturbed
    one on the same X."""
    from oracle import compare as CMP
    rng = np.random.default_rng(seed)
    es, ef = O.RTCURState.eval_subtensor, O.RTCURState.eval_fibers

    def jitter(a):
        return a * (1.0 + rel * rng.standard_normal(a.shape))
    monkeypatch.setattr(O.RTCURState, "eval_subtensor", lambda self, I: jitter(es(self, I)))
    monkeypatch.setattr(O.RTCURState, "eval_fibers", lambda self, d, i, J: jitter(ef(self, d, i, J)))
    try:
        pert = O.rtcur(X, p.ranks, sets, p.zeta0, p.gamma, p.tol, max_iter, variant,
                       keep_full="L" in ref)
    finally:
        monkeypatch.undo()
    n = min(len(pert["hist"]["e"]), len(ref["hist"]["e"]))
    de = float(np.max(np.abs(np.asarray(pert["hist"]["e"][:n]) - np.asarray(ref["hist"]["e"][:n]))))
    if "L" in ref:
        dL = CMP.rel_fro(pert["L"], ref["L"])
    else:  # compare the Tucker states on a seeded grid (no full tensor)
        G = CMP.entry_groups(p.dims, n_slabs=0)[0]
        dL = CMP.rel_fro(pert["state"].eval_subtensor(G), ref["state"].eval_subtensor(G))
    return dL, de
