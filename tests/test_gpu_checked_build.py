"""The bounds-checked build (-DAPIP_CHECK_BOUNDS, libapip_checked.so): it builds,
exports the normal entry points plus apip_check_bounds_selftest, and runs small
cases of every evaluation path (float64 and float32, paper and learned switch,
body order 3 and 4, all-ACE, deterministic mode, MD with list rebuilds) without a
single index out of range, with the forces still at the oracle's parity bars; its
self-test shows that a violation reaches apip_sync as APIP_ERR_BOUNDS.  The cases
run in a child process so that this process keeps the normal library."""
import os
import re
import subprocess
import sys

import pytest

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_runs_clean():
    torch_cuda()
    from paper_2512_07693_gb300 import build
    lib = build.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (apip_\w+)", out))
    header = open(os.path.join(os.path.dirname(HERE), "include", "apip.h")).read()
    for name in set(re.findall(r"\b(apip_[a-z_]+)\s*\(", header)):
        assert name in exported, name
    env = dict(os.environ, APIP_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_child.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "CHECKED OK" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])
