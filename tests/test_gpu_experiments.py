"""The Sec. 4.1 experiment drivers on the CUDA path (GPU only), at a small size: the
phase-transition sweep (batched solves, success = ||L* - L||_F / ||L*||_F <= 1e-3) recovers the
easy corner (low corruption, upsilon = 3) and reports an unsupported cell when |I_i| exceeds the
library's limit; the runtime sweep times whole solves that reach the tolerance (at d = 40 and 64
the recovery itself is not reliable, so only convergence of e^(k) is asserted)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as ge
    ge.build()


def test_phase_transition_small():
    from paper_2108_10448_gb300 import experiments as ex
    out = ex.phase_transition(d=200, ranks=(2, 16), alphas=(0.05, 0.9), upsilons=(3,), trials=3,
                              variants=("F", "R"))
    cells = {(c["variant"], c["r"], c["alpha"]): c for c in out["cells"]}
    for var in ("F", "R"):
        assert cells[(var, 2, 0.05)]["solved"] == 3        # easy corner: every trial recovered
        assert cells[(var, 2, 0.9)]["solved"] == 0         # 90% corruption: none
        assert "unsupported" in cells[(var, 16, 0.05)]     # |I_i| = min(ceil(3 * 16 * ln 200), 200) > 192


def test_runtime_sweep_small():
    from paper_2108_10448_gb300 import experiments as ex
    out = ex.runtime_vs_d(ds=(40, 64), trials=2)
    assert len(out["rows"]) == 4
    for row in out["rows"]:  # every timed solve reached e < 1e-5
        assert row["ms_median"] > 0 and row["iters_median"] > 0 and row["converged"] == 2
