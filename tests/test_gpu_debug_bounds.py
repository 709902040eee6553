"""The FPP_DEBUG_BOUNDS build of libfpp (checks of every gather and scatter
index of the candidate path on the device, the access skipped and the call
failed on a violation; the memory checker is not available on this machine)
runs the parity cases of tests/debug_bounds_run.py without a violation."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_bounds_build_runs_parity_without_a_violation():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_01382_gb300 import _build
    _build.build()
    env = dict(os.environ, FPP_LIBRARY=_build.LIB_DEBUG)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_bounds_run.py")],
                       env=env, capture_output=True, text=True, timeout=600)
    print(r.stdout[-2000:], r.stderr[-2000:])
    assert r.returncode == 0
    assert "no bounds violation" in r.stdout
