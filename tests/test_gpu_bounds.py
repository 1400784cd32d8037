"""The bounds-checked build (compile flag GMMSP_CHECK_BOUNDS): every EM entry point on small
cases, with every launch variant, meets no out-of-range index and still matches the oracle.
The checked library runs in a child process (tests/bounds_cases.py) so that this process keeps
the ordinary one."""
import json
import os
import subprocess
import sys

import pytest

from tests import parity

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_records_no_violation_and_keeps_parity():
    from paper_1612_08792_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, GMMSP_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_cases.py")], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["library"] == lib
    assert len(res["cases"]) == 12 + 8 + 2
    for c in res["cases"]:
        assert c["checked"] is True, c
        assert c["violation"] is None, c
        if "mean_err" in c:
            assert c["mean_err"] <= parity.MEAN_TOL, c
            assert c["agree"] >= parity.LABEL_AGREE and c["worst_margin"] < parity.MARGIN_TOL, c
