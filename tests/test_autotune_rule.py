"""The batched-form autotuner's selection rule on the CPU: the timed probes are replaced by a fake
that returns prescribed times, statuses and recovery counts per (upsilon, cluster), so the rule
itself is checked: candidates below the configured sampling constant are not tried, a candidate
counts only if every problem converges, with known L* only those recovering as many problems as
the best candidate remain, the fastest of those wins, and failures to run are recorded."""
import pytest
import torch

from paper_2108_10448_gb300 import autotune as AT
from paper_2108_10448_gb300 import rtcur as rt


class _Res:
    def __init__(self, status, iters):
        self.status = status
        self.iters = iters


def _install(monkeypatch, spec):
    """spec[(u, c)] = (ms, all_converged, recovered) or an exception instance."""
    last = {}

    def fake_time_batch(X, dims, ranks, zeta0s, gamma, tol, max_iter, variant, u, c, seed, L_out=None):
        last["key"] = (u, c)
        v = spec[(u, c)]
        if isinstance(v, Exception):
            raise v
        ms, ok, _ = v
        return ms, [_Res(rt.OK if ok else rt.NOT_CONVERGED, 10), _Res(rt.OK, 12)]

    def fake_recovered(L_out, L_star, thresh=1e-3):
        return spec[last["key"]][2]

    monkeypatch.setattr(AT, "time_batch", fake_time_batch)
    monkeypatch.setattr(AT, "_recovered", fake_recovered)


def _batch():
    X = [torch.zeros(4, 4, 4), torch.zeros(5, 4, 4)]
    return X, [(4, 4, 4), (5, 4, 4)], [(2, 2, 2), (2, 2, 2)], [1.0, 1.0]


def test_fastest_converged_candidate_wins(monkeypatch):
    spec = {(3.0, 4): (10.0, True, 2), (3.0, 8): (7.0, True, 2), (3.0, 16): (5.0, False, 2),
            (4.0, 4): (9.0, True, 2), (4.0, 8): (8.0, True, 2), (4.0, 16): (6.5, True, 2)}
    _install(monkeypatch, spec)
    X, dims, ranks, z = _batch()
    out = AT.tune_batch(X, dims, ranks, z, clusters=(4, 8, 16), upsilons=(2.0, 3.0, 4.0))
    # (3, 16) is fastest but one problem did not converge; v = 2 is below the configured 3
    assert (out["upsilon"], out["cluster"], out["ms"]) == (4.0, 16, 6.5)
    skipped = [r for r in out["table"] if "skipped" in r]
    assert len(skipped) == 1 and skipped[0]["upsilon"] == 2.0
    assert len([r for r in out["table"] if "ms" in r]) == 6


def test_recovery_outranks_speed(monkeypatch):
    spec = {(3.0, 4): (10.0, True, 2), (3.0, 8): (7.0, True, 1),
            (4.0, 4): (12.0, True, 2), (4.0, 8): (11.0, True, 2)}
    _install(monkeypatch, spec)
    X, dims, ranks, z = _batch()
    L_star = [torch.zeros_like(x) for x in X]
    out = AT.tune_batch(X, dims, ranks, z, clusters=(4, 8), upsilons=(3.0, 4.0), L_star=L_star)
    # (3, 8) is fastest but recovers one problem fewer than the best candidates
    assert (out["upsilon"], out["cluster"]) == (3.0, 4)
    assert all("recovered" in r for r in out["table"])


def test_errors_are_recorded_and_no_converged_candidate_raises(monkeypatch):
    spec = {(3.0, 2): rt.RTCURError(rt.EINVAL, "refine_cluster 2 cannot run for these sample sizes"),
            (3.0, 4): (5.0, False, 0)}
    _install(monkeypatch, spec)
    X, dims, ranks, z = _batch()
    with pytest.raises(RuntimeError):
        AT.tune_batch(X, dims, ranks, z, clusters=(2, 4), upsilons=(3.0,))
    spec[(3.0, 4)] = (5.0, True, 0)
    out = AT.tune_batch(X, dims, ranks, z, clusters=(2, 4), upsilons=(3.0,))
    assert out["cluster"] == 4
    assert any("error" in r and r["cluster"] == 2 for r in out["table"])


def test_results_are_cached_by_signature(monkeypatch, tmp_path):
    spec = {(3.0, 4): (5.0, True, 0), (3.0, 8): (4.0, True, 0)}
    _install(monkeypatch, spec)
    X, dims, ranks, z = _batch()
    path = str(tmp_path / "tune.json")
    out1 = AT.tune_batch(X, dims, ranks, z, clusters=(4, 8), upsilons=(3.0,), cache_path=path)
    spec[(3.0, 8)] = (9.0, True, 0)  # a second call must come from the cache, not the probes
    out2 = AT.tune_batch(X, dims, ranks, z, clusters=(4, 8), upsilons=(3.0,), cache_path=path)
    assert out1["cluster"] == out2["cluster"] == 8
