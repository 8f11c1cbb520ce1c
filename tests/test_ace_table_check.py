"""CPU test of the host check that apip_create runs on the ACE tables before
any device work: the tables of several bases (streamed, body order <= 3, and
pool, body order 4, among them the cracked slab's n8 / l4 / nu4 basis) pass it,
and a single corrupted key or range of each kind fails it.  The harness
(ace_table_check.cu) is compiled with the library's table builder; no device
code runs."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2512_07693_gb300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def test_ace_table_check(tmp_path):
    if not os.path.exists(NVCC):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "ace_table_check")
    cmd = [NVCC, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC, "-x", "cu",
           os.path.join(ROOT, "tests", "ace_table_check.cu"), os.path.join(CSRC, "ace_tables.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = dict(l.split() for l in out.stdout.splitlines())
    assert len([k for k in lines if "_valid_" in k]) == 8
    assert len([k for k in lines if "_valid_" not in k]) == 16
    failed = [k for k, v in lines.items() if v != "ok"]
    assert not failed, failed
