"""The debug build (build(debug=True): device invariant checks on) gives the
same detection, scores and spectra, bit for bit, as the release build, with no
check failing. Each build runs in its own child process (tests/debug_build_probe.py)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_probe(lib):
    env = dict(os.environ, DDHF_LIB=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_build_probe.py")],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_matches_release_with_no_failed_check():
    from paper_2603_08386_gb300 import build
    rel = build.build()
    dbg = build.build(debug=True)
    a, b = run_probe(rel), run_probe(dbg)
    for k in a:
        assert b[k]["flags"] == 0 and b[k]["status"] == 0, b[k]
        assert a[k] == b[k]
    assert any(len(v["boxes"]) > 0 for v in a.values())
