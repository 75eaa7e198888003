"""The team path (one barrier per frame) that SK_WARP_SLICE=0 selects for one-item
launches, against the oracle: the parity cases of the time-major vector path and
of the grouped input-major path run again in a child process with the switch set
(it is read once per process)."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_team_path_parity():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    env = dict(os.environ, SK_WARP_SLICE="0")
    sel = ("fast_path_shapes or input_major_fast_path or input_major_maximum "
           "or full_array_workload_sampled or full_array_input_major_sampled")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu",
                        "-p", "no:cacheprovider", os.path.join(HERE, "test_parity_gpu.py"),
                        "-k", sel],
                       env=env, cwd=os.path.dirname(HERE), capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
