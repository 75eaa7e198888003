"""The kernels' one bounded device-side wait, made to run out.

Warps of a frame's team on the warp-slice paths combine their parts through a
ring of shared-memory slots; a warp a whole ring ahead waits for its slot, at
most a bounded number of polls, then sets the plan's error word and returns
(no trap, no unbounded spin).  sk_selftest_slot_wait runs that very wait
(wi_commit) against a slot that is never freed.  The checks: the kernel
returns, the plan's next call reports SK_ERR_TIMEOUT once, and the plan (and a
fresh one) then runs bit-exact against the oracle.  The paper has no failure
model; this covers the library's own error path.
"""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402

pytestmark = pytest.mark.gpu

N, M, F = 2048, 256, 40


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda:0")


def _flag(plan, d_in, dev):
    skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
    mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
    sk.sk_flag(plan, d_in, F, skv, mask)
    torch.cuda.synchronize()
    return skv.cpu().numpy(), mask.cpu().numpy()


def _check(got, want):
    assert np.array_equal(got[1], want["mask"])
    assert np.array_equal(got[0].view(np.uint32), want["sk"].view(np.uint32))


@pytest.mark.parametrize("spin_limit", [1, 64, 1 << 22])
def test_slot_wait_runs_out_and_is_reported_once(spin_limit):
    dev = _dev()
    rng = np.random.default_rng(spin_limit)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    want = oracle.flag(x, M, N, 3.0, 0.0)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    plan = sk.sk_plan_create(N, M, 3.0, 0.0)
    try:
        _check(_flag(plan, d_in, dev), want)
        t0 = time.perf_counter()
        assert sk.sk_selftest_slot_wait(plan, spin_limit)
        took = time.perf_counter() - t0
        # the default bound (2^22 polls 64 ns apart) gives up in about a quarter second
        assert took < 10.0, took
        with pytest.raises(sk.SkError) as e:
            _flag(plan, d_in, dev)
        assert e.value.status == sk.SK_ERR_TIMEOUT
        assert "bounded wait" in e.value.message
        # reported once; the plan's next launch runs normally
        _check(_flag(plan, d_in, dev), want)
    finally:
        sk.sk_plan_destroy(plan)
    plan = sk.sk_plan_create(N, M, 3.0, 0.0)
    try:
        _check(_flag(plan, d_in, dev), want)
    finally:
        sk.sk_plan_destroy(plan)


def test_slot_wait_limits_are_checked():
    _dev()
    plan = sk.sk_plan_create(256, 256, 3.0, 0.0)
    try:
        for bad in (0, -1, (1 << 22) + 1):
            with pytest.raises(sk.SkError) as e:
                sk.sk_selftest_slot_wait(plan, bad)
            assert e.value.status == sk.SK_ERR_INVALID_ARG
    finally:
        sk.sk_plan_destroy(plan)
