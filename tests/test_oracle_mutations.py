"""The oracle's pins catch planted mistakes.

Each mutant of ``oracle_mutants.MUTANTS`` (a dropped term, a wrong sign, a
wrong index or offset, a transposed operand, a wrong constant, planted in the
oracle's own source on the CPU) is run in a child pytest process against the
unmodified pin file it names; that file must fail.  A control run with the
plugin loaded and no mutant must pass, so a failure is the mutant's doing.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

from oracle import _native

import oracle_mutants

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(mutant, pin_file):
    env = dict(os.environ)
    env["ORACLE_MUTANT"] = mutant
    env["PYTHONPATH"] = os.pathsep.join([ROOT, HERE, env.get("PYTHONPATH", "")])
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-s", "-p", "oracle_mutants",
           "-p", "no:cacheprovider", "-m", "not gpu", os.path.join(HERE, pin_file)]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return p.returncode, p.stdout + p.stderr


@pytest.fixture(scope="module")
def outcomes():
    _native.build()  # the real tracer, built once before the children start
    names = sorted(oracle_mutants.MUTANTS)
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        futs = {n: ex.submit(_run, n, oracle_mutants.MUTANTS[n][0]) for n in names}
        return {n: f.result() for n, f in futs.items()}


@pytest.mark.parametrize("pin_file", ["test_oracle_radon.py"])
def test_control_run_passes(pin_file):
    rc, out = _run("", pin_file)
    assert rc == 0, out[-2000:]


@pytest.mark.parametrize("mutant", sorted(oracle_mutants.MUTANTS))
def test_pins_catch_the_mutant(outcomes, mutant):
    rc, out = outcomes[mutant]
    assert "oracle mutant planted: %s" % mutant in out, out[-2000:]
    assert rc == 1, "mutant %s survived the pins (rc %d):\n%s" % (mutant, rc, out[-2000:])
