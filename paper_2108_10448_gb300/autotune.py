"""Autotuner for the batched form (rtcur_solve_batched).

It picks two knobs for a batch of problems by timing the batch itself (one graph launch per
probe, device time from CUDA events, after one untimed launch that builds the cached graph):

  * the tile shape of the FP64 pinv refinement: thread-block-cluster CTAs per mode
    (options.refine_cluster in {2, 4, 8, 16}). Many concurrent problems compete for clusters,
    so the best size of a batch is not the best size of one problem alone;
  * the sample-size factor upsilon of the sampling schedule, m_i = ceil(upsilon r_i ln d_i) and
    q_i = ceil(upsilon r_i ln prod_{j != i} d_j) (Sec. 3.4's |I_i|, |J_i|): fewer samples make
    each iteration cheaper but may need more iterations or fail to converge.

A configuration counts only if every problem of the batch reaches the tolerance (status OK).
Reaching the tolerance is measured on the sample and does not prove recovery, and a smaller
upsilon tolerates fewer outliers (Sec. 4.1's phase transition), so speed must not buy a lower
upsilon: candidates below ``min_upsilon`` (the caller's configured sampling constant) are not
tried, and when the planted low-rank tensors are known (``L_star``) a candidate must also recover
as many problems (||L - L*||_F / ||L*||_F <= 1e-3, Sec. 4.1's success criterion) as the best
candidate does. The fastest qualifying one is returned with the whole table, and cached in a JSON
file keyed by the batch's shape signature when ``cache_path`` is given. Host logic only: every
timed step runs in librtcur.so."""
from __future__ import annotations

import hashlib
import json
import os

from . import rtcur as rt
from . import synth


def _signature(dims, ranks, variant, tol, max_iter):
    h = hashlib.sha1(json.dumps([list(map(list, dims)), list(map(list, ranks)), variant, tol,
                                 max_iter]).encode()).hexdigest()
    return h[:16]


def _plans(dims, ranks, zeta0s, gamma, tol, max_iter, variant, upsilon, cluster):
    plans = []
    sizes = []
    try:
        for d, r, z in zip(dims, ranks, zeta0s):
            m, q = synth.sample_sizes(d, r, upsilon)
            sizes.append((m, q))
            plans.append(rt.rtcur_create(d, r, m, q, z, gamma, tol, max_iter,
                                         rt.VARIANT_R if variant == "R" else rt.VARIANT_F,
                                         rt.make_options(refine_cluster=cluster)))
    except rt.RTCURError:
        for p in plans:
            rt.rtcur_destroy(p)
        raise
    return plans, sizes


def time_batch(X, dims, ranks, zeta0s, gamma=0.7, tol=1e-5, max_iter=100, variant="R",
               upsilon=3.0, cluster=0, seed=0, repeats=2, L_out=None):
    """Device time (ms, median of ``repeats``) of one batched solve of the problems with device
    tensors X[b] (L^(k) of each problem into the device tensors L_out[b] when given); returns
    (ms, results)."""
    import torch
    plans, sizes = _plans(dims, ranks, zeta0s, gamma, tol, max_iter, variant, upsilon, cluster)
    try:
        n_sets = max_iter if variant == "R" else 1
        idx = [synth.pack_index_sets(synth.draw_index_sets(d, m, q, seed=seed + b, n_sets=n_sets))
               for b, (d, (m, q)) in enumerate(zip(dims, sizes))]
        stream = torch.cuda.current_stream()
        xp = [x.data_ptr() for x in X]
        lp = [l.data_ptr() for l in L_out] if L_out is not None else None
        res = rt.rtcur_solve_batched(plans, xp, idx, lp, None, stream.cuda_stream, max_iter=max_iter)
        times = []
        for _ in range(repeats):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = rt.rtcur_solve_batched(plans, xp, idx, None, None, stream.cuda_stream, max_iter=max_iter)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        times.sort()
        return times[len(times) // 2], res
    finally:
        for p in plans:
            rt.rtcur_destroy(p)


def _recovered(L_out, L_star, thresh=1e-3):
    """Problems whose L is within relative Frobenius ``thresh`` of the planted L* (Sec. 4.1)."""
    import torch
    n = 0
    for L, Ls in zip(L_out, L_star):
        d = torch.linalg.vector_norm((L - Ls).double()) / torch.linalg.vector_norm(Ls.double())
        n += int(float(d) <= thresh)
    return n


def tune_batch(X, dims, ranks, zeta0s, gamma=0.7, tol=1e-5, max_iter=100, variant="R",
               clusters=(2, 4, 8, 16), upsilons=(3.0,), seed=0, cache_path=None, min_upsilon=3.0,
               L_star=None):
    """Returns {"cluster", "upsilon", "ms", "table"} for the fastest qualifying configuration:
    every problem converges, upsilon >= min_upsilon and, with L_star (device tensors of the
    planted low-rank parts), as many problems recovered as by the best candidate."""
    import torch
    sig = _signature(dims, ranks, variant, tol, max_iter) + f"-u{min_upsilon:g}" + ("-L" if L_star else "")
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if sig in cache:
            return cache[sig]
    table = []
    L_out = [torch.empty_like(x) for x in X] if L_star is not None else None
    for u in upsilons:
        if u < min_upsilon:
            table.append({"upsilon": u, "skipped": f"below the configured sampling constant {min_upsilon:g}"})
            continue
        for c in clusters:
            try:
                ms, res = time_batch(X, dims, ranks, zeta0s, gamma, tol, max_iter, variant, u, c, seed,
                                     L_out=L_out)
            except rt.RTCURError as exc:
                table.append({"upsilon": u, "cluster": c, "error": str(exc)})
                continue
            ok = all(r.status == rt.OK for r in res)
            row = {"upsilon": u, "cluster": c, "ms": ms, "converged": ok,
                   "iters": int(sum(r.iters for r in res))}
            if L_star is not None:
                row["recovered"] = _recovered(L_out, L_star)
            table.append(row)
    rows = [r for r in table if r.get("converged")]
    if L_star is not None and rows:
        most = max(r["recovered"] for r in rows)
        rows = [r for r in rows if r["recovered"] == most]
    if not rows:
        raise RuntimeError("no configuration converged on every problem")
    best = min(rows, key=lambda r: r["ms"])
    out = {"cluster": best["cluster"], "upsilon": best["upsilon"], "ms": best["ms"], "table": table}
    if cache_path:
        cache[sig] = out
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return out
