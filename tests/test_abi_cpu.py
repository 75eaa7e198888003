"""The C ABI without a GPU: the library loads, exports every symbol that
include/sk.h declares, and its host-only pieces behave."""

import ctypes
import os
import re

import numpy as np
import pytest

import paper_1808_10365_b300 as sk
from oracle import digitisation as dg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sk.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sk_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = sk.library()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(sk.EXPORTED) == names


def test_digitisation_offset_matches_oracle_model():
    for s in (0.7, 1.0, 1.52, 2.0, 2.5, 3.0, 3.5, 10.0):
        assert abs(sk.sk_digitisation_offset(s) - float(dg.delta_of_sigma(s))) < 1e-12
    with pytest.raises(sk.SkError) as e:
        sk.sk_digitisation_offset(-1.0)
    assert e.value.status == sk.SK_ERR_INVALID_ARG


def test_argument_errors_are_status_codes():
    lib = sk.library()
    out = ctypes.c_void_p(123)
    assert lib.sk_plan_create(None, 0, ctypes.byref(out)) == sk.SK_ERR_INVALID_ARG
    assert out.value is None
    assert "NULL" in sk.sk_last_error()
    p, _ = sk._params(0, 256, 3.0, 0.0, 0, 0, None)
    assert lib.sk_plan_create(ctypes.byref(p), 0, ctypes.byref(out)) == sk.SK_ERR_INVALID_ARG
    p, _ = sk._params(256, 1, 3.0, 0.0, 0, 0, None)
    assert lib.sk_plan_create(ctypes.byref(p), 0, ctypes.byref(out)) == sk.SK_ERR_INVALID_ARG
    p, _ = sk._params(256, 256, -1.0, 0.0, 0, 0, None)
    assert lib.sk_plan_create(ctypes.byref(p), 0, ctypes.byref(out)) == sk.SK_ERR_INVALID_ARG
    assert lib.sk_compute(None, None, 1, None, None, None, None, None, None) == \
        sk.SK_ERR_INVALID_ARG
    assert lib.sk_flag(None, None, 0, None, None, None) == sk.SK_ERR_INVALID_ARG
    assert lib.sk_batch_create(None, 0, 0, ctypes.byref(out)) == sk.SK_ERR_INVALID_ARG
    assert lib.sk_ticket_wait(None, 1, 0, None, None) == sk.SK_ERR_INVALID_ARG
    assert lib.sk_plan_destroy(None) == sk.SK_OK
    assert lib.sk_server_destroy(None) == sk.SK_OK


def test_no_device_is_an_error_not_a_crash():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(sk.SkError) as e:
        sk.sk_plan_create(256, 256)
    assert e.value.status in (sk.SK_ERR_CUDA, sk.SK_ERR_INVALID_ARG)


def test_binding_rejects_buffers_before_any_call():
    """Buffer checks of the binding: size against the plan's N and M, contiguity, and
    host versus device memory.  They raise before the library is called (the plan
    handle here is fake and must never reach it)."""
    import torch

    fake = 0x5EED
    sk._plan_shape[fake] = (256, 256)
    try:
        F = 2
        need = F * 256 * 256
        cases = [
            # device calls given host memory
            lambda: sk.sk_flag(fake, np.zeros(need, np.uint8), F, None, np.zeros(F, np.uint8)),
            lambda: sk.sk_flag(fake, torch.zeros(need, dtype=torch.uint8), F, None, None),
            lambda: sk.sk_compute(fake, np.zeros(need, np.uint8), F),
            # host calls: too small, not contiguous
            lambda: sk.sk_flag_host(fake, np.zeros(need - 1, np.uint8), F, None,
                                    np.zeros(F, np.uint8)),
            lambda: sk.sk_flag_host(fake, np.zeros(need, np.uint8), F, np.zeros(1, np.float32),
                                    np.zeros(F, np.uint8)),
            lambda: sk.sk_flag_host(fake, np.zeros((F, 2 * 256 * 256), np.uint8)[:, ::2], F,
                                    None, np.zeros(F, np.uint8)),
            lambda: sk.sk_flag_host_noalloc(fake, np.zeros(need, np.uint8), F, None,
                                            np.zeros(F - 1, np.uint8)),
        ]
        for k, call in enumerate(cases):
            with pytest.raises(sk.SkError) as e:
                call()
            assert e.value.status == sk.SK_ERR_INVALID_ARG, k
        sk._stream_shape[(fake, 3)] = (256, 256)
        with pytest.raises(sk.SkError):
            sk.sk_stream_submit(fake, 3, np.zeros(256 * 255, np.uint8))
    finally:
        sk._plan_shape.pop(fake, None)
        sk._stream_shape.pop((fake, 3), None)


def test_autotune_cache_lines_merge(tmp_path):
    """The tuner's cache file: one 9-field line per shape (sk_launch_config_t order),
    a shape's new line replacing its old one, other shapes kept."""
    from paper_1808_10365_b300 import autotune

    path = tmp_path / "tiles.txt"
    path.write_text("# old\n2048 256 0 16 0\n256 256 0 16 0\n")
    e = dict(N=2048, M=256, layout=0, rows=16, grid_ctas=0, path=1, team_log2=0, prefetch=1,
             batch_path=2)
    autotune.write_cache(str(path), [e])
    lines = [ln.split() for ln in path.read_text().splitlines() if not ln.startswith("#")]
    assert ["256", "256", "0", "16", "0"] in lines
    assert ["2048", "256", "0", "16", "0", "1", "0", "1", "2"] in lines
    assert sum(1 for ln in lines if ln[:3] == ["2048", "256", "0"]) == 1
    cands = autotune.candidates(2048, 256, 0, 0)
    assert cands[0]["path"] == 0 and len(cands) == 1 + 2 * (3 + 1)
    assert len(autotune.candidates(2048, 256, 1, 8)) == 1 + 3 * 2 * 2
    # small frames also try the stream path (with and without the L2 prefetch)
    small = autotune.candidates(100, 100, 0, 0)
    assert [c["prefetch"] for c in small if c["path"] == sk.SK_PATH_STREAM] == [0, 1]
    assert not [c for c in autotune.candidates(2047, 256, 0, 0) if c["path"] == sk.SK_PATH_STREAM]
