"""The checked build (libbdc_checks.so, the same sources compiled with
-DBDC_CHECKS): every guarded index is tested against the extent of its array
and a failure is recorded as BDC_ECHECK instead of an access out of range.
The same workload (tests/checked_run.py: single-pass, split, stepped and
streaming sweeps, the literal walks, exact channels, certificate, divergence,
dual bound, counts, the allocation-free marginal) runs under both builds in
child processes; no check fires, and the results are the same."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def _run(checked):
    env = dict(os.environ)
    env["BDC_CHECKED"] = "1" if checked else "0"
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def _flat(v):
    if isinstance(v, dict):
        return [x for k in sorted(v) if k != "lib" for x in _flat(v[k])]
    if isinstance(v, list):
        return [x for e in v for x in _flat(e)]
    return [float(v)]


def test_checked_build_runs_clean_and_agrees():
    from paper_2604_05867_b300 import build
    build.build(checks=True)
    rel = _run(False)
    chk = _run(True)
    assert chk["lib"].endswith("libbdc_checks.so") and rel["lib"].endswith("libbdc.so")
    a, b = np.array(_flat(rel)), np.array(_flat(chk))
    assert a.shape == b.shape
    assert np.all(np.abs(a - b) <= 1e-13 * np.maximum(1.0, np.abs(a)))
