"""The library built with index bound checks (QSIM_DEBUG) on the small
parity cases: plain sweeps of every kind, staged tiles, the QFT in
complex128.  Runs in a process of its own (QSIM_LIBRARY=debug)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_small_parity_cases():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2203_08826_gb300 import build
    build.build(debug=True)
    env = dict(os.environ, QSIM_LIBRARY="debug")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_build_cases.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 indices outside the state" in r.stdout
