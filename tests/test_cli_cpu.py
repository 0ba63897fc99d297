"""The command-line drivers import and parse their options without a GPU (a syntax or import
error in a driver would otherwise surface only on the GPU machine)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("args", [
    ["bench.py", "--help"],
    ["-m", "paper_1511_04552_gb300.warmstart", "--help"],
    ["-m", "paper_1511_04552_gb300.studies", "--help"],
])
def test_driver_help(args):
    r = subprocess.run([sys.executable] + args, cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    assert "usage:" in r.stdout
