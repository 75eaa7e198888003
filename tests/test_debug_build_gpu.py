"""The debug build of the library (-DSK_DEBUG, libsk_debug.so): its kernels check
every global load and store against the item's buffers and report a failed check
through the plan's error word instead of trapping.  In a child process (the binding
loads the debug build when SK_DEBUG_LIBRARY=1): small cases of every read path are
exact against the oracle with no check failing; and with the input taken as one
byte shorter than it is (SK_DEBUG_SHRINK_INPUT=1) the last load fails its check, is
skipped, and the plan's next call reports it -- no fault, no trap."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(os.path.dirname(HERE), "paper_1808_10365_b300", "libsk_debug.so")


def _run(args, extra_env):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    if not os.path.exists(LIB):
        pytest.fail("libsk_debug.so not built (paper_1808_10365_b300/build.py)")
    # the built-in launch configurations, not the tuned cache: the child checks
    # which path each case takes
    env = dict(os.environ, SK_DEBUG_LIBRARY="1", SK_AUTOTUNE_CACHE="", **extra_env)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_child.py")] + args,
                       env=env, capture_output=True, text=True, timeout=600)
    print(r.stdout[-2000:], r.stderr[-4000:])
    return r


def test_debug_build_every_path_exact_and_no_check_fails():
    r = _run([], {})
    assert r.returncode == 0
    assert "every case exact" in r.stdout


def test_debug_build_reports_a_failed_bounds_check():
    r = _run(["shrink"], {"SK_DEBUG_SHRINK_INPUT": "1"})
    assert r.returncode == 0
    assert "bounds check reported" in r.stdout
