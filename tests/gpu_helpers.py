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


def support_mismatch(S_gpu, ref, X, band_rel=1e-6):
    """Support differences between the GPU's S^(k) and the oracle's, split into entries inside
    the band ||X - L^(k-1)| - zeta| <= band_rel * zeta (allowed) and outside it (not allowed)."""
    zeta = ref["zeta"]
    D = X.astype(np.float64) - ref["prev_state"].full(X.shape)
    band = np.abs(np.abs(D) - zeta) <= band_rel * zeta
    diff = (S_gpu != 0) != (ref["S"] != 0)
    return int(np.count_nonzero(diff & band)), int(np.count_nonzero(diff & ~band))
