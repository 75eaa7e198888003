"""The paths that switches select for one-item launches, against the oracle: the
team path (one barrier per frame, SK_WARP_SLICE=0) and the warp-slice path
handing out whole frames (SK_ROW_BALANCE=0).  The parity cases of the time-major
vector path and of the grouped input-major path run again in a child process
with the switch set (switches are read once per process)."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("switch", ["SK_WARP_SLICE", "SK_ROW_BALANCE"])
def test_switched_path_parity(switch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    env = dict(os.environ, **{switch: "0"})
    sel = ("fast_path_shapes or input_major_fast_path or input_major_maximum "
           "or full_array_workload_sampled or full_array_input_major_sampled")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu",
                        "-p", "no:cacheprovider", os.path.join(HERE, "test_parity_gpu.py"),
                        "-k", sel],
                       env=env, cwd=os.path.dirname(HERE), capture_output=True, text=True,
                       timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
