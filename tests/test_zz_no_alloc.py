"""sk_flag_host_noalloc: the host-buffer flagging call for callers that must not
allocate device memory once running (their HBM belongs to another allocator, or
an allocation could stall a real-time loop).  It must give exactly what the
oracle and sk_flag_host give -- masks and SK bit for bit, the bar of every
parity test here -- call after call, on a fresh plan (no row-balancing scratch
yet: whole frames per team) as well as on one that has its scratch, leave the
device's free memory unchanged, and refuse requests larger than its fixed
staging area.  Collected last on purpose."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402
import synth  # noqa: E402
from oracle import digitisation as dg  # noqa: E402

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


def test_noalloc_first_on_a_fresh_plan_matches_oracle_and_allocates_nothing():
    """The call as its users make it: a plan created at start-up, then only this
    call.  With no earlier sk_flag_host the plan has no row-balancing scratch, so
    the launch hands whole frames to the teams; after an sk_flag_host call has
    allocated the scratch, it balances rows.  Both against the oracle, and the
    device's free memory (cudaMemGetInfo) the same before and after every call."""
    _need_gpu()
    N, M = 2048, 256
    ds = synth.full_array_config(n_freq=1, n_frames=60, N=N, M=M, cfg=9)[0]
    x = ds.generate_cpu()
    delta = float(np.mean(dg.delta_of_sigma(ds.sigma)))
    parts = [np.ascontiguousarray(x[:30]), np.ascontiguousarray(x[30:53]),
             np.ascontiguousarray(x[:30])]
    wants = [oracle.flag(p, M, N, 3.0, delta) for p in parts]
    plan = sk.sk_plan_create(N, M, 3.0, delta)
    try:
        torch.cuda.synchronize()
        free = [torch.cuda.mem_get_info()[0]]
        for p, w in zip(parts, wants):
            got_sk, got_mask = _noalloc(plan, p, p.shape[0])
            free.append(torch.cuda.mem_get_info()[0])
            assert np.array_equal(got_mask, w["mask"])
            assert np.array_equal(got_sk.view(np.uint32), w["sk"].view(np.uint32))
        print("free device memory around the calls:", free)
        assert len(set(free)) == 1, free
        # sk_flag_host allocates the plan's scratch; the call then balances rows
        _reference(plan, parts[0], parts[0].shape[0])
        for p, w in zip(parts, wants):
            got_sk, got_mask = _noalloc(plan, p, p.shape[0])
            assert np.array_equal(got_mask, w["mask"])
            assert np.array_equal(got_sk.view(np.uint32), w["sk"].view(np.uint32))
    finally:
        sk.sk_plan_destroy(plan)


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
