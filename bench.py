"""Benchmark of the GB300 RTCUR hot path (one JSON line on stdout, rank 0).

A step is one RTCUR iteration (Algorithm 1's loop body) on the 800^3 rank-5 workload: the
sampled threshold + gather, the FP64 truncated pinv, the factor update, the sampled stopping
error and, in the FULL scope (default), the dense fused threshold pass over the whole 2 GB
tensor. `value` is iterations/s with X resident in HBM (X is 2.05 GB, larger than L2, so no
flush is needed between iterations). Extra keys: the dense kernel's roofline (timed live with
CUDA events on the stream it runs on), time to e <= 1e-5, an end-to-end number through the
C ABI with host buffers, and the FP64 oracle timed on the host cores as the CPU baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--scope full|sampled] [--variant F|R] [--size D]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RTCUR iters/s & time-to-1e-5 at 800³ rank 5: BF16/TF32 vs FP32 plain, % HBM roofline"


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal bandwidth (context for the roofline fraction)

# DRAM bytes (read + write) of one launch of the FP32 fused dense pass k_dense_tma<5,0,1>, from an
# ncu capture of two back-to-back launches at 600^3 without cache control (the second launch: the
# dirty lines the first left in L2 are written back inside it, as its own are after it), scaled
# by the element count. None until that capture exists; must be dropped whenever the kernel
# changes.
DENSE_TRAFFIC_PER_ELEMENT = 1734200064.0 / 216e6  # 8.029 B per element
DENSE_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of k_dense_tma<5,0,1>, 600^3, "
                        "second of two back-to-back launches, --cache-control none, scaled by elements "
                        "(profiles/k_dense_tma_traffic_600.md)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scope", default="full", choices=["full", "sampled"])
    ap.add_argument("--variant", default="F", choices=["F", "R"])
    ap.add_argument("--size", type=int, default=800)
    ap.add_argument("--rank", type=int, default=5)
    ap.add_argument("--alpha", type=float, default=0.3)
    ap.add_argument("--upsilon", type=float, default=3.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the per-form comparison")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-form comparison (64 uneven problems)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing")
    ap.add_argument("--quick", action="store_true",
                    help="only the timed iterations and the dense kernel's roofline (for profiling runs)")
    return ap.parse_args()


def workload_name(a):
    return (f"RTCUR-{a.variant} {a.scope.upper()} scope, {a.size}^3 FP32 Gaussian Tucker rank "
            f"({a.rank},{a.rank},{a.rank}), {int(a.alpha * 100)}% outliers U[-10 mean|L*|, 10 mean|L*|], "
            f"v={a.upsilon:g}, gamma=0.7, zeta0=max|X|, tol 1e-5")


def workload_config(a, p, world=1):
    """The workload's description, identical in both arms' JSON lines."""
    return {"workload": workload_name(a), "dims": list(p.dims), "ranks": list(p.ranks), "nI": p.m,
            "nJ": p.q, "variant": a.variant, "scope": a.scope,
            "l2": (f"inputs larger than L2 (X is {p.X.nbytes / 1e9:.2f} GB, L2 0.13 GB), no flush"
                   if p.X.nbytes > 2 * 129e6 else "inputs smaller than L2 (a small case, not a bench figure)"),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def make_problem(a):
    from paper_2108_10448_gb300 import synth
    p = synth.make_tucker_problem((a.size,) * 3, (a.rank,) * 3, a.alpha, a.upsilon, seed=a.seed,
                                  keep_truth=False, max_iter=100)
    n_sets = 100 if a.variant == "R" else 1
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=a.seed, n_sets=n_sets)
    return p, sets


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class OracleFull:
    """Algorithm 1 in the FULL scope, one iteration per ``step()``, run by the FP64 oracle as it
    stands: the decay, Step (I) over the whole tensor (L^(k) formed in full by the literal chain,
    HT, the residual), then the sampled step (gather, Fiber CUR with LAPACK SVD, e^(k+1))."""

    def __init__(self, p, sets, variant):
        from oracle import rtcur_oracle as O
        self.O = O
        self.p, self.sets, self.variant = p, sets, variant
        self.Xd = p.X.astype(np.float64)  # set-up (the oracle works in FP64)
        self.st = O.RTCURState()
        self.zeta = p.zeta0
        self.k = 0

    def step(self):
        O, p = self.O, self.p
        self.zeta *= p.gamma
        s = self.sets[0] if self.variant == "F" else self.sets[self.k % len(self.sets)]
        D = self.Xd - self.st.full(p.dims)
        S = O.hard_threshold(D, self.zeta)
        resid = float(np.sum((D - S) ** 2))
        del D, S
        self.st, info = O.rtcur_step(self.Xd, self.st, s, self.zeta, p.ranks)
        self.k += 1
        return resid, info["e"]


def oracle_full_iterations(p, sets, variant, n_untimed, n_timed):
    """Wall time of ``n_timed`` whole FULL-scope oracle iterations after ``n_untimed`` (the first
    iteration, with L^(0) = 0, is cheaper than the rest)."""
    orc = OracleFull(p, sets, variant)
    for _ in range(n_untimed):
        orc.step()
    times = []
    for _ in range(n_timed):
        t0 = time.perf_counter()
        orc.step()
        times.append(time.perf_counter() - t0)
    return times


def oracle_sampled_solve(p, sets, variant):
    """The oracle's whole SAMPLED-scope solve to tol (Sec. 3.3's partial S update: the paper's
    efficient form), timed; returns (seconds, result)."""
    from oracle import rtcur_oracle as O
    t0 = time.perf_counter()
    ref = O.rtcur(p.X, p.ranks, sets, p.zeta0, p.gamma, p.tol, p.max_iter, variant)
    return time.perf_counter() - t0, ref


def oracle_parity(p, sets, variant, gpu, ref, form_s=None):
    """The GPU solve's results (host copies at the comparison entries, ``gather_for_oracle``)
    against the oracle's solve ``ref``: iterations, histories, L, and the support of S split into
    in-band / L-explained / unexplained differences. ``form_s`` maps other dense forms to their S
    at the same entries (same iterates, only the dense pass differs)."""
    from oracle import compare as CMP
    k = ref["iters"]
    out = {"iters_gpu": gpu["iters"], "iters_oracle": k, "iters_equal": gpu["iters"] == k}
    if gpu["iters"] != k or k == 0:
        return out
    last = sets[0] if variant == "F" else sets[k - 1]
    groups = CMP.entry_groups(p.dims)
    assert all(all(np.array_equal(a, b) for a, b in zip(G, H)) for G, H in zip(groups, gpu["groups"]))
    orc = CMP.oracle_values(ref, p.dims, last, groups)
    z = np.asarray(ref["hist"]["zeta"])
    e = np.asarray(ref["hist"]["e"])
    out["zeta_max_rel_diff"] = float(np.max(np.abs(gpu["zeta_hist"] - z) / z))
    out["e_max_abs_diff"] = float(np.max(np.abs(gpu["e_hist"] - e)))
    out["e_max_rel_diff"] = float(np.max(np.abs(gpu["e_hist"] - e) / np.maximum(e, 1e-300)))
    rel, fl = CMP.compare_entries(p.X, groups, orc, gpu["L_sample"], gpu["L_groups"], gpu["S_groups"],
                                  gpu["Lprev_groups"], ref["zeta"])
    out["rel_L"] = rel
    out["support"] = fl
    out["entries"] = ("L: every sampled entry of the last iteration + a seeded 100^3 grid + 4 "
                      "mode-1 slabs; S: the grid and the slabs")
    if form_s:
        # a reduced-precision dense pass evaluates L^(k-1) itself: its flips are L-explained within
        # the form's evaluation error (relative to max|L|), the same bands as the GPU form tests
        band = {"fp32_plain": 2e-6, "bf16": 1e-4, "tf32": 4e-3, "fp32_compressed_S": 0.0}
        maxL = max(float(np.max(np.abs(v))) for v in orc["Lprev_groups"])
        out["forms"] = {}
        for name, Sg in form_s.items():
            _, f2 = CMP.compare_entries(p.X, groups, orc, gpu["L_sample"], gpu["L_groups"], Sg,
                                        gpu["Lprev_groups"], ref["zeta"], extra=band[name] * maxL)
            out["forms"][name] = dict(f2, evaluation_band=f"{band[name]:g} max|L|")
    return out


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(a, rank, world):
    """The reference arm: the FP64 oracle as it stands on the host cores, one whole FULL-scope
    iteration of the same workload per step (W untimed, then K timed; nothing extrapolated)."""
    if rank != 0:
        return
    p, sets = make_problem(a)
    K, W = a.steps, a.warmup
    times = oracle_full_iterations(p, sets, a.variant, W, K)
    t = float(np.sum(times))
    value = K / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": t / K * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(a, p, world),
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"{K} whole FULL-scope oracle iterations ({W + 1}..{W + K}) of the "
                                   f"workload after {W} untimed ones, each timed; numpy elementwise "
                                   "steps run on one core, LAPACK/BLAS on all"},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def aggregate_replicas(ms, K, world, device="cpu"):
    """Replicas: the timed region's duration is the max over ranks, and the job's value is the
    iterations of all ranks over it. Collective only for N > 1 (an initialised process group)."""
    if world > 1:
        import torch
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
        torch.distributed.barrier()
    return ms, world * K / (ms / 1e3)


def run_batched(dev):
    """Batched form on 64 uneven 3-mode problems (dims U{64..320}, ranks U{2..10}, outliers
    10-40%, RTCUR-R, v = 3, tol 1e-5): 64 sequential rtcur_solve calls against one
    rtcur_solve_batched graph launch with the same plans, then the autotuned configuration."""
    import torch
    from paper_2108_10448_gb300 import autotune
    from paper_2108_10448_gb300 import rtcur as rt
    from paper_2108_10448_gb300 import synth
    probs = synth.make_batched_problems(64)
    X = [torch.from_numpy(p.X).to(dev) for p in probs]
    idx = [synth.pack_index_sets(synth.draw_index_sets(p.dims, p.m, p.q, seed=b, n_sets=p.max_iter))
           for b, p in enumerate(probs)]
    plans = [rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, p.max_iter,
                             rt.VARIANT_R, rt.make_options()) for p in probs]
    s = torch.cuda.current_stream(dev).cuda_stream
    xp = [x.data_ptr() for x in X]
    try:
        for b, pl in enumerate(plans):  # warm: builds each plan's graphs
            rt.rtcur_solve(pl, xp[b], idx[b], 0, 0, s, max_iter=probs[b].max_iter)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seq = [rt.rtcur_solve(pl, xp[b], idx[b], 0, 0, s, max_iter=probs[b].max_iter)
               for b, pl in enumerate(plans)]
        torch.cuda.synchronize()
        seq_s = time.perf_counter() - t0
        rt.rtcur_solve_batched(plans, xp, idx, None, None, s, max_iter=100)  # builds the graph
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bat = rt.rtcur_solve_batched(plans, xp, idx, None, None, s, max_iter=100)
        torch.cuda.synchronize()
        bat_s = time.perf_counter() - t0
    finally:
        for pl in plans:
            rt.rtcur_destroy(pl)
    same = all(x.iters == y.iters and x.e == y.e for x, y in zip(seq, bat))
    # the tuner times the refinement cluster size at the workload's own v = 3 (and v = 4): it may
    # not lower v for speed, and every candidate must recover as many planted L* as the best
    Ls = [torch.from_numpy(p.L_star.astype(np.float32)).to(dev) for p in probs]
    tuned = autotune.tune_batch(X, [p.dims for p in probs], [p.ranks for p in probs],
                                [p.zeta0 for p in probs], variant="R", tol=1e-5, max_iter=100,
                                upsilons=(3.0, 4.0), min_upsilon=3.0, L_star=Ls)
    del Ls
    return {
        "workload": "64 uneven 3-mode FP32 problems, dims U{64..320}, ranks U{2..10}, outliers "
                    "U[10%, 40%], RTCUR-R, v=3, tol 1e-5 (seeds 0..63)",
        "elements": int(sum(p.X.size for p in probs)),
        "sequential_s": seq_s, "batched_s": bat_s, "speedup": seq_s / bat_s,
        "problems_per_s_batched": len(probs) / bat_s,
        "iters_total": int(sum(r.iters for r in bat)),
        "all_converged": all(r.status == rt.OK for r in bat),
        "batched_equals_sequential": same,
        "tuned": {"cluster": tuned["cluster"], "upsilon": tuned["upsilon"],
                  "graph_ms": tuned["ms"], "table": tuned["table"],
                  "rule": "fastest of the candidates at v >= 3 that converge on every problem and "
                          "recover (||L - L*||/||L*|| <= 1e-3) as many problems as the best"},
        "timing": "wall clock around the public calls (index upload, graph launch, results)",
    }


def run_adjoint(dev):
    """Adjoint workload: K = 10 unrolled RTCUR-F iterations on 200^3, rank (5,5,5), 20% outliers;
    device time of the forward (with checkpoints) and of rtcur_backward."""
    import torch
    from paper_2108_10448_gb300 import rtcur as rt
    from paper_2108_10448_gb300 import synth
    K = 10
    p = synth.make_tucker_problem((200, 200, 200), (5, 5, 5), 0.2, 3.0, seed=0, keep_truth=True)
    sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=0)
    idx = synth.pack_index_sets(sets)
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, 0.0, K, rt.VARIANT_F,
                           rt.make_options(checkpoint=K))
    X = torch.from_numpy(p.X).to(dev)
    L = torch.empty_like(X)
    dL = torch.empty_like(X)
    dX = torch.empty_like(X)
    Ls = torch.from_numpy(p.L_star.astype(np.float32)).to(dev)
    st = torch.cuda.current_stream(dev)
    s = st.cuda_stream
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    fw, bw = [], []
    try:
        for rep in range(4):
            e0.record(st)
            rt.rtcur_begin(plan, X.data_ptr(), idx, 0, s)
            rt.rtcur_iterate(plan, K, s)
            rt.rtcur_finish(plan, L.data_ptr(), 0, s, max_iter=K)
            e1.record(st)
            torch.mul(torch.sub(L, Ls), 2.0, out=dL)
            rt.rtcur_backward(plan, dL.data_ptr(), dX.data_ptr(), s)
            e2.record(st)
            torch.cuda.synchronize()
            if rep:
                fw.append(e0.elapsed_time(e1))
                bw.append(e1.elapsed_time(e2))
    finally:
        rt.rtcur_destroy(plan)
    return {"workload": "K=10 unrolled RTCUR-F, 200^3 FP32, rank (5,5,5), 20% outliers, "
                        "loss ||L_K - L*||_F^2",
            "forward_ms": float(np.median(fw)), "backward_ms": float(np.median(bw)),
            "includes": "forward: begin + 10 iterations + L materialisation; backward: "
                        "seed dL + rtcur_backward (FP64 pinv adjoints)"}


def take(T, coords):
    """Host FP64 copy of a device tensor's entries at integer coordinate arrays."""
    import torch
    idx = tuple(torch.from_numpy(np.ascontiguousarray(np.asarray(c).reshape(-1))).to(T.device) for c in coords)
    return T[idx].cpu().numpy().astype(np.float64).reshape(np.asarray(coords[0]).shape)


def comparison_coords(p, sets, variant, iters):
    """Coordinates the oracle comparison reads: the last iteration's sampled entries (R, then the
    fibers) and the entry groups (a seeded 100^3 grid and 4 mode-1 slabs). Built without the
    oracle: the same recipe as the comparison's own groups (checked there by shape)."""
    rng = np.random.default_rng(1234)
    dims = p.dims
    groups = [[np.sort(rng.choice(int(d), size=min(int(d), 100), replace=False)) for d in dims]]
    for s0 in np.sort(rng.choice(int(dims[0]), size=min(int(dims[0]), 4), replace=False)):
        groups.append([np.array([s0])] + [np.arange(int(d)) for d in dims[1:]])
    last = sets[0] if variant == "F" else sets[max(iters - 1, 0) % len(sets)]
    samp = [np.meshgrid(*last["I"], indexing="ij")]
    for i in range(len(dims)):
        rest = int(np.prod([d for j, d in enumerate(dims) if j != i]))
        J = np.asarray(last["J"][i])
        rem = J.copy()
        oc = [None] * len(dims)
        for l in reversed(range(len(dims))):
            if l == i:
                continue
            oc[l] = rem % dims[l]
            rem = rem // dims[l]
        assert rest > 0
        samp.append([np.broadcast_to(np.arange(dims[i])[:, None], (dims[i], J.size)) if l == i else
                     np.broadcast_to(oc[l][None, :], (dims[i], J.size)) for l in range(len(dims))])
    return groups, samp


def gather_for_oracle(p, sets, variant, res, L, S, Lprev):
    """Host copies of a GPU solve's results at the comparison entries."""
    groups, samp = comparison_coords(p, sets, variant, res.iters)
    grids = [np.meshgrid(*G, indexing="ij") for G in groups]
    return {"groups": groups, "iters": res.iters, "e_hist": np.asarray(res.e_hist),
            "zeta_hist": np.asarray(res.zeta_hist),
            "L_sample": np.concatenate([take(L, c).ravel() for c in samp]),
            "L_groups": [take(L, c) for c in grids], "S_groups": [take(S, c) for c in grids],
            "Lprev_groups": [take(Lprev, c) for c in grids]}


def solve_timed(rt, plan, X, idx, L, S, sh, stream, max_iter, reps=7, skip=2):
    """Whole solves from X resident (index upload, max|X|, the graph-driven loop, L and S output):
    CUDA-event times of ``reps`` solves, the first ``skip`` untimed; returns (median ms, all, last res)."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ts, res = [], None
    for rep in range(reps):
        ev0.record(stream)
        res = rt.rtcur_solve(plan, X.data_ptr(), idx, L.data_ptr() if L is not None else 0,
                             S.data_ptr() if S is not None else 0, sh, max_iter=max_iter)
        ev1.record(stream)
        torch.cuda.synchronize()
        if rep >= skip:
            ts.append(ev0.elapsed_time(ev1))
    return float(np.median(ts)), ts, res


def iterations_timed(rt, plan, X, idx, S, sh, stream, K, W):
    """W untimed then K timed iterations (rtcur_iterate), CUDA events on the launching stream."""
    import torch
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    rt.rtcur_begin(plan, X.data_ptr(), idx, S.data_ptr() if S is not None else 0, sh)
    rt.rtcur_iterate(plan, W, sh)
    torch.cuda.synchronize()
    ev0.record(stream)
    rt.rtcur_iterate(plan, K, sh)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def run_ours(a, rank, world):
    import torch
    from paper_2108_10448_gb300 import rtcur as rt
    from paper_2108_10448_gb300 import synth
    import __graft_entry__ as ge

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0 or world == 1:
        ge.build()
    if world > 1:
        torch.distributed.barrier()
    rt.load()
    p, sets = make_problem(a)
    idx = synth.pack_index_sets(sets)
    X = torch.from_numpy(p.X).to(dev)
    L = torch.empty_like(X)
    S = torch.empty_like(X)
    scope = rt.SCOPE_FULL if a.scope == "full" else rt.SCOPE_SAMPLED
    variant = rt.VARIANT_R if a.variant == "R" else rt.VARIANT_F
    max_iter = 100
    plan = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter, variant,
                           rt.make_options(scope=scope))
    stream = torch.cuda.Stream(device=dev)
    sh = stream.cuda_stream
    K, W = a.steps, a.warmup
    # --- iterations/s: W warm-up iterations, then K timed, device-timed with events ---
    rt.rtcur_begin(plan, X.data_ptr(), idx, S.data_ptr(), sh)
    rt.rtcur_iterate(plan, W, sh)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        rt.rtcur_iterate(plan, K, sh)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms, value = aggregate_replicas(ev0.elapsed_time(ev1), K, world, dev)
    rt.rtcur_finish(plan, 0, 0, sh, max_iter=max_iter)
    N = int(np.prod(p.dims))
    # --- dominant kernel alone: the dense fused pass, same launch configuration ---
    roof = None
    if scope == rt.SCOPE_FULL:
        rt.rtcur_threshold_dense(plan, 3, sh)
        torch.cuda.synchronize()
        nl = 10
        ev0.record(stream)
        rt.rtcur_threshold_dense(plan, nl, sh)
        ev1.record(stream)
        torch.cuda.synchronize()
        dms = ev0.elapsed_time(ev1) / nl
        alg_bytes = 8.0 * N  # 4 B read of X + 4 B write of S per element
        peak, src = peaks()
        achieved = alg_bytes / (dms / 1e3) / 1e9
        traffic = (DENSE_TRAFFIC_PER_ELEMENT * N
                   if DENSE_TRAFFIC_PER_ELEMENT is not None and p.ranks[-1] == 5 else None)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "traffic_source": DENSE_TRAFFIC_SOURCE if traffic is not None else None,
                "kernel": f"k_dense_tma<{p.ranks[-1]},0,{int(p.dims[-1] <= 2048)}>", "ms_per_launch": dms,
                "peak_source": f"{src} (burst copy bandwidth); the >= 0.70 target refers to it",
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                "iteration_frac": alg_bytes / (ms / K / 1e3) / 1e9 / peak,
                "algorithmic_bytes_per_launch": alg_bytes}
    if a.quick:
        rt.rtcur_destroy(plan)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
                              "steps": K, "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
                              "quick": True, "config": workload_config(a, p, world), "roofline": roof}),
                  flush=True)
        return
    # --- time to tolerance: whole solve from X resident, one graph launch; median of 5 after 2 ---
    ttt_ms, ttts, res = solve_timed(rt, plan, X, idx, L, S, sh, stream, max_iter)
    parity_gpu = {}
    want_parity = rank == 0 and not a.no_cpu_baseline and res.iters >= 1
    if want_parity:
        Lprev = torch.empty_like(X)
        pp = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max(res.iters - 1, 1),
                             variant, rt.make_options(scope=scope))
        if res.iters > 1:
            rt.rtcur_solve(pp, X.data_ptr(), idx, Lprev.data_ptr(), 0, sh, max_iter=res.iters - 1)
        else:
            Lprev.zero_()
        rt.rtcur_destroy(pp)
        torch.cuda.synchronize()
        parity_gpu[a.variant] = gather_for_oracle(p, sets, a.variant, res, L, S, Lprev)
        del Lprev
    # --- dense-pass forms: same iterates, different evaluation of L in the dense pass ---
    forms_out, form_S = None, {}
    if scope == rt.SCOPE_FULL and not a.no_forms:
        forms_out = {}
        groups, _ = comparison_coords(p, sets, a.variant, res.iters)
        grids = [np.meshgrid(*G, indexing="ij") for G in groups]
        for name, form, sfmt in (("fp32_plain", rt.FORM_FP32_PLAIN, rt.S_DENSE), ("bf16", rt.FORM_BF16, rt.S_DENSE),
                                 ("tf32", rt.FORM_TF32, rt.S_DENSE),
                                 ("fp32_compressed_S", rt.FORM_FP32, rt.S_COMPRESSED)):
            try:
                fp = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter,
                                     variant, rt.make_options(scope=scope, dense_form=form, s_format=sfmt))
            except rt.RTCURError as exc:
                forms_out[name] = {"unavailable": str(exc)}
                continue
            Sf = torch.empty_like(X)
            fms = iterations_timed(rt, fp, X, idx, Sf, sh, stream, K, W)
            rt.rtcur_threshold_dense(fp, 2, sh)
            torch.cuda.synchronize()
            ev0.record(stream)
            rt.rtcur_threshold_dense(fp, 5, sh)
            ev1.record(stream)
            torch.cuda.synchronize()
            dms_f = ev0.elapsed_time(ev1) / 5
            fbytes, extra = 8.0 * N, {}
            if sfmt == rt.S_COMPRESSED:
                c = rt.rtcur_get_s_compressed(fp, sh)
                # read X, write the nonzero values and the mask words
                fbytes = 4.0 * N + 4.0 * c["nnz"] + 4.0 * c["rows"] * c["words_per_row"]
                extra = {"nnz": c["nnz"], "bytes_per_element": fbytes / N}
            # whole solve to tolerance with this form: S^(k) of the final iterate
            f_ttt, _, fres = solve_timed(rt, fp, X, idx, None, Sf, sh, stream, max_iter, reps=3, skip=1)
            if sfmt == rt.S_COMPRESSED:
                extra["S_bit_equal_to_fp32"] = bool(torch.equal(Sf, S))
            mism = int(((Sf != 0) != (S != 0)).sum().item())
            if want_parity and fres.iters == res.iters:
                form_S[name] = [take(Sf, c) for c in grids]
            rt.rtcur_destroy(fp)
            del Sf
            forms_out[name] = {"iters_per_s": K / (fms / 1e3), "ms_per_iter": fms / K,
                               "dense_ms": dms_f, "dense_gbs": fbytes / (dms_f / 1e3) / 1e9,
                               "time_to_tol_ms": f_ttt, "iters": fres.iters,
                               "S_support_mismatch_vs_fp32_final": mism, **extra}
        forms_out["fp32_fused"] = {"iters_per_s": value / world, "ms_per_iter": ms / K,
                                   "dense_ms": roof["ms_per_launch"] if roof else None,
                                   "time_to_tol_ms": ttt_ms, "iters": res.iters}
        forms_out["note"] = ("every form runs the same CUR iterates (the sampled chain is FP32/FP64 in "
                             "all of them); only the dense pass's evaluation of L, hence S near the "
                             "threshold, differs. S support against the oracle: support_vs_oracle.forms")
    # --- the other variant at the same workload (RTCUR-R when the main line is F, and back) ---
    other = "R" if a.variant == "F" else "F"
    var_out = None
    if world == 1:
        o_sets = synth.draw_index_sets(p.dims, p.m, p.q, seed=a.seed, n_sets=100 if other == "R" else 1)
        o_idx = synth.pack_index_sets(o_sets)
        ov = rt.VARIANT_R if other == "R" else rt.VARIANT_F
        op = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter, ov,
                             rt.make_options(scope=scope))
        oms = iterations_timed(rt, op, X, o_idx, S, sh, stream, K, W)
        o_ttt, o_ts, ores = solve_timed(rt, op, X, o_idx, L, S, sh, stream, max_iter)
        rt.rtcur_destroy(op)
        var_out = {"variant": other, "iters_per_s": K / (oms / 1e3), "ms_per_iter": oms / K,
                   "time_to_tol": {"ms": o_ttt, "runs_ms": o_ts, "iters": ores.iters, "e": ores.e,
                                   "status": ores.status}}
        if want_parity and ores.iters >= 1:
            Lprev = torch.empty_like(X)
            pp = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol,
                                 max(ores.iters - 1, 1), ov, rt.make_options(scope=scope))
            if ores.iters > 1:
                rt.rtcur_solve(pp, X.data_ptr(), o_idx, Lprev.data_ptr(), 0, sh, max_iter=ores.iters - 1)
            else:
                Lprev.zero_()
            rt.rtcur_destroy(pp)
            torch.cuda.synchronize()
            parity_gpu[other] = gather_for_oracle(p, o_sets, other, ores, L, S, Lprev)
            del Lprev
    # --- SAMPLED scope (the paper's efficient form, Sec. 3.3): time to 1e-5, both variants ---
    sampled_ttt = {}
    if world == 1:
        for v in ("F", "R"):
            v_sets = sets if v == a.variant else synth.draw_index_sets(
                p.dims, p.m, p.q, seed=a.seed, n_sets=100 if v == "R" else 1)
            sp_ = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter,
                                  rt.VARIANT_R if v == "R" else rt.VARIANT_F,
                                  rt.make_options(scope=rt.SCOPE_SAMPLED))
            v_ms, v_ts, vres = solve_timed(rt, sp_, X, synth.pack_index_sets(v_sets), L, None, sh, stream, max_iter)
            rt.rtcur_destroy(sp_)
            sampled_ttt[v] = {"ms": v_ms, "runs_ms": v_ts, "iters": vres.iters, "e": vres.e,
                              "status": vres.status}
            # the same solve with the sampled step reading a BF16 copy of X (option sample_x)
            bp = rt.rtcur_create(p.dims, p.ranks, p.m, p.q, p.zeta0, p.gamma, p.tol, max_iter,
                                 rt.VARIANT_R if v == "R" else rt.VARIANT_F,
                                 rt.make_options(scope=rt.SCOPE_SAMPLED, sample_x=rt.SAMPLE_X_BF16))
            b_ms, _, bres = solve_timed(rt, bp, X, synth.pack_index_sets(v_sets), L, None, sh, stream,
                                        max_iter, reps=4, skip=1)
            rt.rtcur_destroy(bp)
            sampled_ttt[v]["sample_x_bf16"] = {"ms": b_ms, "iters": bres.iters, "e": bres.e,
                                               "note": "includes the BF16 copy of X made by rtcur_begin"}
    # --- end to end through the C ABI from pinned host buffers: H2D X, the solve, and the
    # download of Algorithm 1's output (R, C_i, U_i^+, from which L = R x_i (C_i U_i^+)); beside
    # it the same solve with the dense L^(K) downloaded instead (the host link, ~0.2 TB/s each way,
    # then takes as long as the solve)
    Xh = torch.from_numpy(p.X).pin_memory()
    Lh = torch.empty_like(Xh).pin_memory()
    Xd = torch.empty_like(X)
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        Xd.copy_(Xh, non_blocking=True)
        res_e2e = rt.rtcur_solve(plan, Xd.data_ptr(), idx, 0, 0, sh, max_iter=max_iter)
        cur = rt.rtcur_get_cur(plan, p.dims, p.m, p.q, sh)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_val = world * res_e2e.iters / e2e_s
    cur_bytes = int(cur[0].nbytes + sum(c.nbytes for c in cur[1]) + sum(u.nbytes for u in cur[2]))
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        Xd.copy_(Xh, non_blocking=True)
        res_l = rt.rtcur_solve(plan, Xd.data_ptr(), idx, L.data_ptr(), 0, sh, max_iter=max_iter)
        Lh.copy_(L, non_blocking=True)
    torch.cuda.synchronize()
    e2e_l_s = time.perf_counter() - t0
    rt.rtcur_destroy(plan)
    del Xd, Xh, Lh
    if rank != 0:
        return
    n_modes = 3
    # per iteration: [dense pass] + threshold + Gram + warm refinement + eigensolver + refinement
    # + B_i (partials, reduce) + one core stage per mode + table (2) + error + commit
    launches_per_iter = (1 if scope == rt.SCOPE_FULL else 0) + 1 + 1 + 1 + 1 + 1 + 2 + n_modes + 2 + 1 + 1
    line = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(a, p, world),
        "implementation": {"dense_form": "fp32 fused (FMA last-mode product)", "pinv": "fp64"},
        "time_to_tol": {"ms": ttt_ms, "runs_ms": ttts, "iters": res.iters, "e": res.e, "status": res.status,
                        "warm_hits": res.warm_hits, "statistic": "median of 5 solves after 2 warm-up solves",
                        "includes": "index upload, max|X|, the graph-driven loop, L and S output"},
        "e2e": {"value": e2e_val, "unit": "iters/s", "seconds": e2e_s, "iters": res_e2e.iters,
                "h2d_bytes_per_step": int(p.X.nbytes) + int(idx.nbytes), "d2h_bytes_per_step": cur_bytes,
                "step": "one whole solve: H2D X (and the index sets), rtcur_solve to 1e-5, D2H of "
                        "Algorithm 1's output R, C_i, U_i^+ (rtcur_get_cur)",
                "dense_L": {"value": world * res_l.iters / e2e_l_s, "seconds": e2e_l_s,
                            "d2h_bytes_per_step": int(p.X.nbytes),
                            "step": "the same with the dense L (prod d_i floats) downloaded instead"}},
        "roofline": roof,
        "other_variant": var_out,
        "sampled_time_to_tol": sampled_ttt or None,
        "forms": forms_out,
        "gpu_launches": launches_per_iter * K,
        "clocks": clk.summary(),
    }
    del X, L, S
    torch.cuda.empty_cache()
    line["batched"] = None if (a.no_batched or world > 1) else run_batched(dev)
    line["adjoint"] = None if (a.no_adjoint or world > 1) else run_adjoint(dev)
    if not a.no_cpu_baseline:
        # the oracle as it stands on the host cores: two whole FULL-scope iterations of the
        # workload (after one untimed), then its SAMPLED-scope solves to tol, whose results are
        # also compared with the GPU's
        t_full = oracle_full_iterations(p, sets, a.variant, 1, 2)
        line["cpu_baseline"] = {
            "value": len(t_full) / float(np.sum(t_full)), "unit": "iters/s", "cores": cpu_cores(),
            "kind": "oracle",
            "sample": "2 whole FULL-scope iterations (2 and 3) of the workload by the FP64 oracle, "
                      "each timed, nothing extrapolated; numpy elementwise steps on one core, "
                      "LAPACK/BLAS on all",
            "iteration_s": t_full}
        orc_ttt, support = {}, {}
        for v in ("F", "R"):
            v_sets = sets if v == a.variant else synth.draw_index_sets(
                p.dims, p.m, p.q, seed=a.seed, n_sets=100 if v == "R" else 1)
            t_or, ref = oracle_sampled_solve(p, v_sets, v)
            orc_ttt[v] = {"s": t_or, "iters": ref["iters"], "e": ref["e"],
                          "gpu_sampled_ms": sampled_ttt.get(v, {}).get("ms"),
                          "speedup": (t_or * 1e3 / sampled_ttt[v]["ms"]) if v in sampled_ttt else None}
            if v in parity_gpu:
                support[v] = oracle_parity(p, v_sets, v, parity_gpu[v], ref,
                                           form_S if v == a.variant else None)
            del ref
        line["cpu_baseline"]["sampled_solve_to_tol"] = orc_ttt
        line["cpu_baseline"]["sampled_note"] = ("the oracle's SAMPLED-scope solve to 1e-5 (the paper's "
                                                "efficient method), beside the GPU's SAMPLED-scope "
                                                "time to 1e-5 of the same problem and index sets")
        line["support_vs_oracle"] = support
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch
        backend = "nccl" if a.impl == "ours" else "gloo"
        torch.distributed.init_process_group(backend)
    try:
        if a.impl == "reference":
            run_reference(a, rank, world)
        else:
            run_ours(a, rank, world)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
