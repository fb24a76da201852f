"""The bounds-checked build (SA_CHECKED): every computing call runs on small workloads
with every index its kernels take from data range-checked, records no violation, and
gives the plain build's outputs bit for bit.  Each build runs in a fresh process."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(checked: bool):
    env = dict(os.environ, SA_CHECKED="1" if checked else "0")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_records_no_violation_and_matches_the_plain_build(cuda_lib):
    checked, plain = _run(True), _run(False)
    assert checked.pop("checked") is True and plain.pop("checked") is False
    assert checked.pop("status") is None and plain.pop("status") is None
    assert checked.keys() == plain.keys() and len(checked) >= 20
    diff = [k for k in checked if checked[k] != plain[k]]
    assert not diff, diff
