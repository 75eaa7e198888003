"""Input sharding on the GPU: the inputs of one frequency split into shards, each
shard's per-frame Q and N_eff from sk_compute, their exact sums, and sk_finish
with the whole array's plan, against sk_flag on the whole array (bit-identical)
and the oracle; the NCCL helper with a one-rank group; sk_finish's argument and
range checks."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda:0")


def _shard(x, M, N, lo, hi, layout):
    F = x.shape[0]
    if layout == 0:
        return np.ascontiguousarray(x.reshape(F, M, N)[:, :, lo:hi]).reshape(F, -1)
    return np.ascontiguousarray(x.reshape(F, N, M)[:, lo:hi, :]).reshape(F, -1)


@pytest.mark.parametrize("N,M,F,cuts,layout", [
    (2048, 256, 37, [0, 1024, 2048], 0),           # two warp-slice shards
    (2048, 256, 11, [0, 512, 1536, 2048], 1),      # three input-major shards
    (1000, 96, 9, [0, 333, 1000], 0),              # ragged shards: general path
    (4096, 128, 5, [0, 2048, 4096], 0)])
def test_shards_summed_match_whole_array(N, M, F, cuts, layout):
    dev = _dev()
    rng = np.random.default_rng(N + M + F + layout)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    want = oracle.flag(x, M, N, 3.0, 0.03, layout=layout)
    q = torch.zeros(F, dtype=torch.int64, device=dev)
    ne = torch.zeros(F, dtype=torch.int32, device=dev)
    plans = []
    try:
        for lo, hi in zip(cuts[:-1], cuts[1:]):
            xs = torch.from_numpy(_shard(x, M, N, lo, hi, layout).reshape(-1)).to(dev)
            p = sk.sk_plan_create(hi - lo, M, 3.0, 0.03, layout=layout)
            plans.append(p)
            qs = torch.empty(F, dtype=torch.int64, device=dev)
            ns = torch.empty(F, dtype=torch.int32, device=dev)
            sk.sk_compute(p, xs, F, None, None, qs, None, ns)
            q += qs
            ne += ns
        whole = sk.sk_plan_create(N, M, 3.0, 0.03, layout=layout)
        plans.append(whole)
        skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
        mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
        sk.sk_finish(whole, q, ne, F, skv, mask)
        d_in = torch.from_numpy(x.reshape(-1)).to(dev)
        sk2 = torch.empty(F, dtype=torch.float32, device=dev)
        m2 = torch.empty(F, dtype=torch.uint8, device=dev)
        sk.sk_flag(whole, d_in, F, sk2, m2)
        torch.cuda.synchronize()
    finally:
        for p in plans:
            sk.sk_plan_destroy(p)
    assert np.array_equal(q.cpu().numpy(), want["Q"])
    assert np.array_equal(ne.cpu().numpy(), want["neff"])
    assert np.array_equal(mask.cpu().numpy(), want["mask"])
    assert np.array_equal(skv.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32))
    assert np.array_equal(skv.cpu().numpy().view(np.uint32), sk2.cpu().numpy().view(np.uint32))
    assert np.array_equal(mask.cpu().numpy(), m2.cpu().numpy())


def test_flag_sharded_one_rank_nccl_group():
    """The helper end to end with NCCL: a one-rank group, whose all-reduce is the
    identity, gives sk_flag's results."""
    import torch.distributed as dist

    from paper_1808_10365_b300 import sharding

    dev = _dev()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0,
                            world_size=1, device_id=dev)
    try:
        N, M, F = 2048, 256, 29
        rng = np.random.default_rng(77)
        x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
        want = oracle.flag(x, M, N, 3.0, 0.0)
        d_in = torch.from_numpy(x.reshape(-1)).to(dev)
        plan = sk.sk_plan_create(N, M, 3.0, 0.0)
        try:
            skv = torch.empty(F, dtype=torch.float32, device=dev)
            mask = torch.empty(F, dtype=torch.uint8, device=dev)
            st = torch.cuda.Stream(dev)
            sharding.flag_sharded(plan, plan, d_in, F, skv, mask, stream=st)
            torch.cuda.synchronize()
        finally:
            sk.sk_plan_destroy(plan)
        assert np.array_equal(mask.cpu().numpy(), want["mask"])
        assert np.array_equal(skv.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32))
    finally:
        dist.destroy_process_group()


def test_finish_checks():
    dev = _dev()
    plan = sk.sk_plan_create(64, 32, 3.0, 0.0)
    try:
        q = torch.zeros(3, dtype=torch.int64, device=dev)
        ne = torch.tensor([-1, 65, 0], dtype=torch.int32, device=dev)
        skv = torch.zeros(3, dtype=torch.float32, device=dev)
        mask = torch.zeros(3, dtype=torch.uint8, device=dev)
        sk.sk_finish(plan, q, ne, 3, skv, mask)
        sk.sk_finish(plan, q, ne, 0, None, mask)       # nothing to do
        torch.cuda.synchronize()
        assert mask.cpu().tolist() == [1, 1, 1]        # out of range, out of range, no power
        assert np.isnan(skv.cpu().numpy()).all()
        with pytest.raises(sk.SkError) as e:
            sk.sk_finish(plan, q, ne, 3, skv, None)
        assert e.value.status == sk.SK_ERR_INVALID_ARG
    finally:
        sk.sk_plan_destroy(plan)
    running = sk.sk_plan_create(64, 32, 3.0, 0.0, flags=sk.SK_RUNNING_OFFSET)
    try:
        with pytest.raises(sk.SkError) as e:
            sk.sk_finish(running, q, ne, 3, skv, mask)
        assert e.value.status == sk.SK_ERR_UNSUPPORTED
    finally:
        sk.sk_plan_destroy(running)
