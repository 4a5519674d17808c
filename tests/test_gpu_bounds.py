"""The bounds-checked build (compute-sanitizer is not available here): the
library compiled with SPS_BOUNDS_CHECK=1 tests every staged shared-memory read
of the de-dispersion passes (single channels, pre-summed pairs and quads, the
batched work-list form, subband step two) against its stage and records a read
that would leave it in the plan's status word instead of making it.  Every
path, on ragged shapes and on the full beam, must run with a clean status word
and give the oracle's result."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checked_build_runs_clean():
    subprocess.run([sys.executable, "-m", "paper_1811_04165_gb300.build", "--checked"], cwd=ROOT, check=True,
                   capture_output=True, timeout=1200)
    env = dict(os.environ, SPS_BUILD="checked")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_worker.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")]
    assert r.returncode == 0 and line, r.stderr[-3000:]
    res = json.loads(line[0][7:])
    assert len(res) >= 30
    bad = {k: v for k, v in res.items() if v["status"] != 0 or not v["ok"]}
    assert not bad, bad
