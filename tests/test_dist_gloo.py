"""Multi-rank host logic on CPU (gloo, world size 2): bench.py's barrier,
max-over-ranks timing and per-rank frequency sharding (independent seeds, no
data-path collective), and the input-sharding exchange (exact integer sums of
the ranks' per-frame Q and N_eff) checked against the oracle on the whole
array."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, loc = bench.dist_setup()
        bench.barrier(w)
        m = bench.max_over_ranks(1.0 + 2.0 * r, w)
        ds = bench.workload_datasets(r)
        seeds = [d.seed for d in ds]
        x = ds[0].generate_cpu(0, 1)
        q.put((r, w, m, seeds, int(x.sum())))
    finally:
        dist.destroy_process_group()


def test_two_ranks_time_max_and_disjoint_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    out.sort()
    assert [o[1] for o in out] == [2, 2]
    assert out[0][2] == out[1][2] == 3.0           # max over ranks of 1 and 3
    assert set(out[0][3]).isdisjoint(out[1][3])    # each rank its own frequencies
    assert out[0][4] != out[1][4]


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun the reference arm (the oracle on the host) runs on rank 0 alone;
    another rank exits 0 without output."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2",
               MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=root, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=root, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def _shard_worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import numpy as np

    import oracle
    from paper_1808_10365_b300 import sharding

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        N, M, F = 96, 64, 23
        rng = np.random.default_rng(4242)           # every rank draws the whole array
        x = rng.integers(0, 256, size=(F, M, N), dtype=np.uint8)
        x[3, :, :40] = 0x88                          # dead inputs, both shards
        bounds = [0, 40, N][rank:rank + 2]           # uneven shards: 40 and 56 inputs
        mine = np.ascontiguousarray(x[:, :, bounds[0]:bounds[1]])
        n_mine = bounds[1] - bounds[0]
        S1, S2 = oracle.power_sums(mine.reshape(F, -1), M, n_mine)
        Qr, ner, _ = oracle.sk_spec(S1, S2, M)
        qt = torch.from_numpy(np.asarray(Qr, dtype=np.int64).copy())
        nt = torch.from_numpy(np.asarray(ner, dtype=np.int32).copy())
        sharding.exchange_partials(qt, nt)
        whole = oracle.flag(x.reshape(F, -1), M, N, 3.0, 0.01)
        m = oracle.mask(qt.numpy(), nt.numpy(), whole["t_lo"], whole["t_hi"])
        q.put((rank, bool(np.array_equal(qt.numpy(), whole["Q"])),
               bool(np.array_equal(nt.numpy(), whole["neff"])),
               bool(np.array_equal(m, whole["mask"])), int(whole["neff"][3])))
    finally:
        dist.destroy_process_group()


def test_two_ranks_input_sharding_exchange():
    """Two ranks hold 40 and 56 of 96 inputs; after the exchange each has the whole
    array's Q, N_eff and mask exactly."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, q_ok, n_ok, m_ok, neff3 in out:
        assert q_ok and n_ok and m_ok, rank
        assert neff3 == 96 - 40
