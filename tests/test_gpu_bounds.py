"""The bounds-checked build (compute-sanitizer is closed on this machine): every
global access of the FP32 stage kernels checks its offset against its
buffer's extent, and a violation is skipped and reported (SWE_ERR_BOUNDS,
source line in error_cell). No case may report one; and a build told that
the last row of every state plane is out of bounds (the allocation is
untouched, so nothing outside it is ever touched) must report it for every
whole domain and for windows of every decomposition."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
SWE_ERR_BOUNDS = -6


@pytest.fixture(scope="module")
def debug_lib():
    from paper_1912_02457_gb300 import build
    return build.build_debug()


def _run(lib, extra_env=None):
    env = dict(os.environ, SWE_LIBRARY=lib, **(extra_env or {}))
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_no_access_leaves_its_buffer(debug_lib):
    res = _run(debug_lib)
    assert len(res) >= 40
    bad = {k: v for k, v in res.items() if v[0] != 0}
    assert not bad, bad


def test_the_checks_catch_a_shrunk_extent(debug_lib):
    res = _run(debug_lib, {"SWE_DEBUG_SHRINK_PLANE_ROWS": "1"})
    flagged = {k: v for k, v in res.items() if v[0] == SWE_ERR_BOUNDS}
    # every whole domain touches its last row; the reported line lies in the
    # kernel source
    whole = [k for k in res if not k.startswith("split ")]
    assert all(k in flagged for k in whole), {k: res[k] for k in whole if k not in flagged}
    assert all(v[1] > 0 for v in flagged.values())
    # a window plans its wet own rows only, so one whose top rows are all
    # land reads no cell of its last row; every decomposition has windows
    # that do
    splits = {}
    for k in res:
        if k.startswith("split "):
            w = k.split()
            splits.setdefault((w[1], " ".join(w[4:])), []).append(k in flagged)
    assert splits and all(any(v) for v in splits.values()), splits
