"""The paper's two synthetic experiments (Sec. 4.1) run on the CUDA path through the C ABI.

* Phase transition (Fig. 2 protocol): d x d x d tensors, multilinear rank (r, r, r), a fraction
  alpha of entries corrupted; for each (r, alpha, upsilon) and variant, `trials` problems are
  solved in one batched graph launch (`rtcur_solve_batched`) with zeta^(0) = ||L*||_inf,
  gamma = 0.7, tolerance 1e-5, and a problem counts as solved when
  ||L* - L^(k)||_F / ||L*||_F <= 1e-3.
* Runtime versus dimension (Fig. 3 protocol, this method only): rank (3, 3, 3), 10% corruption,
  upsilon = 3, zeta^(0) = ||L*||_inf, gamma = 0.7, halting at e^(k) < 1e-5; the time of one whole
  solve (index upload, the graph-driven loop, L output) averaged over `trials` problems.

Inputs follow the recipe of Sec. 4.1: L* = Y x_1 Y_1 x_2 Y_2 x_3 Y_3 with standard normal core
and factors; the support of S* is a uniformly random set of floor(alpha N) entries, its values
uniform in [-E|L*|, E|L*|] (E|L*| taken as the mean over the tensor). They are drawn on the GPU
with torch's seeded generator (plumbing: a 300^3 problem is generated in milliseconds); the
index sets come from `synth.draw_index_sets` as everywhere else.

Usage: python -m paper_2108_10448_gb300.experiments {phase,runtime} --out results.json [...]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import rtcur as rt
from . import synth


def tucker_problem_gpu(d, r, alpha, seed, device, outlier_scale=1.0):
    """(X, L*) as FP32 CUDA tensors of shape (d, d, d) and zeta^(0) = max|L*|."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    core = torch.randn((r, r, r), generator=g, device=device, dtype=torch.float64)
    Y = [torch.randn((d, r), generator=g, device=device, dtype=torch.float64) for _ in range(3)]
    L = torch.einsum("abc,ia,jb,kc->ijk", core, Y[0], Y[1], Y[2]).contiguous()
    N = d * d * d
    k = int(math.floor(alpha * N))
    scale = outlier_scale * float(L.abs().mean())
    X = L.clone().view(-1)
    if k > 0:
        pos = torch.randperm(N, generator=g, device=device)[:k]
        X[pos] += (torch.rand(k, generator=g, device=device, dtype=torch.float64) * 2.0 - 1.0) * scale
    zeta0 = float(L.abs().max())
    return X.view(d, d, d).float().contiguous(), L.float().contiguous(), zeta0


def _rel_err(L, Ls):
    import torch
    return float(torch.linalg.vector_norm((L - Ls).double()) / torch.linalg.vector_norm(Ls.double()))


def phase_transition(d=300, ranks=(3, 5, 10), alphas=(0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7),
                     upsilons=(1, 2, 3, 4, 5), trials=10, variants=("F", "R"), seed=0, max_iter=100,
                     sampling="fiber", log=None):
    """Success counts per (variant, r, upsilon, alpha). sampling = "fiber" draws J_i uniformly
    (|J_i| = ceil(v r ln d^2)); "chidori" takes J_i = prod_{j != i} I_j (|J_i| = |I|^2). Cells
    whose sample sizes exceed the library's limits are reported as unsupported."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream().cuda_stream
    dims = (d, d, d)
    out = {"d": d, "trials": trials, "alphas": list(alphas), "sampling": sampling, "cells": []}
    t0 = time.time()

    def draw(m, q, sd, n_sets):
        if sampling == "chidori":
            return synth.draw_chidori_sets(dims, m, seed=sd, n_sets=n_sets)
        return synth.draw_index_sets(dims, m, q, seed=sd, n_sets=n_sets)

    for r in ranks:
        # the problems of one (r, alpha) serve every upsilon and variant
        probs = {}
        for ai, a in enumerate(alphas):
            probs[a] = [tucker_problem_gpu(d, r, a, seed * 1000003 + r * 7919 + ai * 101 + t, dev)
                        for t in range(trials)]
        Ls = [torch.empty((d, d, d), device=dev, dtype=torch.float32) for _ in range(trials)]
        for ups in upsilons:
            m, q = synth.sample_sizes(dims, (r, r, r), ups)
            if sampling == "chidori":
                q = [m[1] * m[2], m[0] * m[2], m[0] * m[1]]
            for var in variants:
                cell_base = {"variant": var, "r": r, "upsilon": ups, "m": m[0], "q": q[0]}
                vcode = rt.VARIANT_R if var == "R" else rt.VARIANT_F
                for ai, a in enumerate(alphas):
                    plans = []
                    try:
                        # zeta^(0) = ||L*||_inf is a plan parameter: one plan per problem
                        for X, Lstar, z0 in probs[a]:
                            plans.append(rt.rtcur_create(dims, (r, r, r), m, q, z0, 0.7, 1e-5, max_iter, vcode,
                                                         rt.make_options(scope=rt.SCOPE_SAMPLED)))
                    except rt.RTCURError as exc:  # e.g. |I_i| above the library's limit
                        for pl in plans:
                            rt.rtcur_destroy(pl)
                        out["cells"].append(dict(cell_base, alpha=a, unsupported=str(exc)))
                        continue
                    try:
                        idxs = [synth.pack_index_sets(draw(m, q, seed * 7 + r * 131 + int(ups * 17) + ai * 3 + t,
                                                           max_iter if var == "R" else 1)) for t in range(trials)]
                        res = rt.rtcur_solve_batched(plans, [p[0].data_ptr() for p in probs[a]], idxs,
                                                     L_ptrs=[L.data_ptr() for L in Ls], stream=stream,
                                                     max_iter=max_iter)
                        torch.cuda.synchronize()
                    finally:
                        for pl in plans:
                            rt.rtcur_destroy(pl)
                    errs = [_rel_err(Ls[t], probs[a][t][1]) for t in range(trials)]
                    ok = sum(1 for e in errs if e <= 1e-3)
                    out["cells"].append(dict(cell_base, alpha=a, solved=ok, iters=[int(x.iters) for x in res],
                                             rel_err_median=float(np.median(errs))))
                    if log:
                        log(f"{var} r={r} ups={ups} alpha={a}: {ok}/{trials} "
                            f"(median rel err {np.median(errs):.2e}, {time.time() - t0:.0f} s)")
        del probs
        torch.cuda.empty_cache()
    out["seconds"] = time.time() - t0
    return out


def runtime_vs_d(ds=(100, 200, 300, 400, 500, 600, 700, 800), r=3, alpha=0.1, upsilon=3,
                 trials=10, variants=("F", "R"), seed=0, max_iter=100, log=None):
    """Mean and median time of one whole solve (SAMPLED scope, L output) per d and variant."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.Stream(device=dev)
    sh = st.cuda_stream
    out = {"r": r, "alpha": alpha, "upsilon": upsilon, "trials": trials, "rows": []}
    for d in ds:
        dims = (d, d, d)
        m, q = synth.sample_sizes(dims, (r, r, r), upsilon)
        for var in variants:
            times, iters, errs, conv = [], [], [], 0
            for t in range(trials):
                X, Lstar, z0 = tucker_problem_gpu(d, r, alpha, seed * 1000003 + d * 31 + t, dev)
                idx = synth.pack_index_sets(synth.draw_index_sets(dims, m, q, seed=seed + d + t,
                                                                  n_sets=max_iter if var == "R" else 1))
                plan = rt.rtcur_create(dims, (r, r, r), m, q, z0, 0.7, 1e-5, max_iter,
                                       rt.VARIANT_R if var == "R" else rt.VARIANT_F,
                                       rt.make_options(scope=rt.SCOPE_SAMPLED))
                L = torch.empty_like(X)
                try:
                    # the first solve builds the plan's graphs; the second, identical one is timed
                    rt.rtcur_solve(plan, X.data_ptr(), idx, L.data_ptr(), 0, sh, max_iter=max_iter)
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    res = rt.rtcur_solve(plan, X.data_ptr(), idx, L.data_ptr(), 0, sh, max_iter=max_iter)
                    e1.record(st)
                    torch.cuda.synchronize()
                finally:
                    rt.rtcur_destroy(plan)
                times.append(e0.elapsed_time(e1))
                iters.append(int(res.iters))
                conv += int(res.status == rt.OK)
                errs.append(_rel_err(L, Lstar))
                del X, Lstar, L
            row = {"d": d, "variant": var, "m": m[0], "q": q[0], "ms_mean": float(np.mean(times)),
                   "ms_median": float(np.median(times)), "iters_median": float(np.median(iters)),
                   "converged": conv, "rel_err_median": float(np.median(errs)), "rel_err_max": float(np.max(errs))}
            out["rows"].append(row)
            if log:
                log(json.dumps(row))
            torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("which", choices=["phase", "runtime"])
    ap.add_argument("--out", required=True)
    ap.add_argument("--d", type=int, default=300)
    ap.add_argument("--trials", type=int, default=10)
    ap.add_argument("--ranks", default="3,5,10")
    ap.add_argument("--alphas", default="0.1,0.2,0.3,0.4,0.5,0.6,0.7")
    ap.add_argument("--upsilons", default="1,2,3,4,5")
    ap.add_argument("--ds", default="100,200,300,400,500,600,700,800")
    ap.add_argument("--sampling", default="fiber", choices=["fiber", "chidori"])
    a = ap.parse_args()
    import __graft_entry__ as ge  # builds the library if needed
    ge.build()
    rt.load()

    def log(s):
        print(s, flush=True)

    if a.which == "phase":
        res = phase_transition(d=a.d, ranks=[int(x) for x in a.ranks.split(",")],
                               alphas=[float(x) for x in a.alphas.split(",")],
                               upsilons=[float(x) for x in a.upsilons.split(",")], trials=a.trials,
                               sampling=a.sampling, log=log)
    else:
        res = runtime_vs_d(ds=[int(x) for x in a.ds.split(",")], trials=a.trials, log=log)
    with open(a.out, "w") as f:
        json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
