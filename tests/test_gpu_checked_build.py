"""The checked build on the GPU: the library compiled with SC_BOUNDS_CHECK,
whose traversal verifies every element index it loads or hands to an
epilogue against the item's box, runs the cases of `checked_cases.py` (ragged
tiles, thin and odd boxes, self-periodic boxes, uneven levels, ensembles,
both forms and stagings, the adjoint and the hierarchy).  No check fails --
a failure would raise through the error word -- and every result is bit for
bit the release build's.  This stands in for a device memory checker, which
this GPU pool does not offer."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_checked_build_passes_every_check_and_matches_release():
    from paper_1308_1343_gb300 import build
    checked = build.build(checked=True)
    env = dict(os.environ, SC_LEVEL_LIB=checked)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    import checked_cases
    want = checked_cases.run()
    assert set(got) == set(want)
    for k in want:
        assert got[k] == want[k], k
