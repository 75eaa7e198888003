"""sk_flag_host_noalloc: the host-buffer flagging call for callers that must not
allocate device memory once running (their HBM belongs to another allocator, or
an allocation could stall a real-time loop).  It must give exactly what
sk_flag_host gives -- masks and SK bit for bit, the bar of every parity test
here -- call after call, and refuse requests larger than its fixed staging
area.  Collected last on purpose."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1808_10365_b300 as sk  # noqa: E402
import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def _reference(plan, x, F):
    h_sk = np.zeros(F, dtype=np.float32)
    h_mask = np.zeros(F, dtype=np.uint8)
    sk.sk_flag_host(plan, x, F, h_sk, h_mask)
    return h_sk, h_mask


def _noalloc(plan, x, F):
    h_sk = np.full(F, -1.0, dtype=np.float32)
    h_mask = np.full(F, 7, dtype=np.uint8)
    sk.sk_flag_host_noalloc(plan, x, F, h_sk, h_mask)
    return h_sk, h_mask


def test_noalloc_matches_flag_host_on_consecutive_calls():
    _need_gpu()
    N, M = 2048, 256
    ds = synth.full_array_config(n_freq=1, n_frames=60, N=N, M=M)[0]
    x = ds.generate_cpu()
    delta = float(np.mean([sk.sk_digitisation_offset(s) for s in ds.sigma]))
    plan = sk.sk_plan_create(N, M, 3.0, delta)
    try:
        first = np.ascontiguousarray(x[:30])      # 15.7 MB: fits the fixed area
        second = np.ascontiguousarray(x[30:55])   # a different, smaller request next
        for part in (first, second):
            F = part.shape[0]
            want_sk, want_mask = _reference(plan, part, F)
            got_sk, got_mask = _noalloc(plan, part, F)
            assert np.array_equal(got_mask, want_mask)
            assert np.array_equal(got_sk.view(np.uint32), want_sk.view(np.uint32))
    finally:
        sk.sk_plan_destroy(plan)


def test_noalloc_small_array_and_limits():
    _need_gpu()
    ds = synth.pathfinder_config()
    x = ds.generate_cpu()
    plan = sk.sk_plan_create(256, 256, 3.0, -0.09)
    try:
        for _ in range(2):
            want = _reference(plan, x, 64)
            got = _noalloc(plan, x, 64)
            assert np.array_equal(got[1], want[1])
            assert np.array_equal(got[0].view(np.uint32), want[0].view(np.uint32))
        # 257 frames of 64 KiB are just over the fixed 16 MiB staging area
        big = np.zeros((257, 256 * 256), dtype=np.uint8)
        with pytest.raises(sk.SkError) as e:
            sk.sk_flag_host_noalloc(plan, big, 257, None, np.zeros(257, dtype=np.uint8))
        assert e.value.status == sk.SK_ERR_INVALID_ARG
        assert "staging area" in e.value.message
    finally:
        sk.sk_plan_destroy(plan)
