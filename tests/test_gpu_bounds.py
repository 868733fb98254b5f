"""The bounds-check build (-DRNG_BOUNDS_CHECK, a separate shared object):
tiny and ragged cases of the generation, lagged Fibonacci and Ising kernels
run through it, agree with the oracle, and record no out-of-range shared-
or global-memory index.  The checked build stands in for a memory-checking
tool: every index those kernels compute is compared with its array's extent
before the access."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_tiny_and_ragged_cases_under_the_bounds_check_build():
    import importlib.util
    spec = importlib.util.spec_from_file_location("rng_gb300_build", os.path.join(ROOT, "paper_1204_6193_gb300",
                                                                                   "build.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    lib = b.build(bounds=True)
    env = dict(os.environ, RNG_GB300_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py")], env=env, capture_output=True,
                       text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    print(res)
    assert res["cases"] > 200
    assert res["failed"] == []
    assert res["bounds_site"] == 0, f"out-of-range access recorded at site {res['bounds_site']}"
