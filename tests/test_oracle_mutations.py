"""Mutation test of the oracle pins (CPU): each planted mistake of `oracle_mutants` (a strict >
made non-strict, an inverted singular value, squared norms in e^(k), a reversed fiber decode, no
zeta decay, one singular value too many, the sign of S in R; and in the adjoint a wrong factor 2,
a dropped Daleckii-Krein coupling, inverted masks, a missing fiber term, a sign flip) must make
at least one pin fail. Each mutant runs the pin file in a child process."""
import os
import subprocess
import sys

import pytest

from oracle_mutants import MUTANTS

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    target = "tests/test_oracle_adjoint.py" if MUTANTS[name][0].endswith("adjoint") else "tests/test_oracle_pins.py"
    env = dict(os.environ, RTCUR_ORACLE_MUTANT=name,
               PYTHONPATH=os.pathsep.join([HERE, ROOT, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "oracle_mutants", "-m", "not gpu",
                        "-p", "no:cacheprovider", target], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 1, f"mutant {name} survived or errored (exit {r.returncode}):\n{r.stdout[-1500:]}"
