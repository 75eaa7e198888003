"""Plans shared across host threads: sk_flag on one plan from several threads, each
on its own CUDA stream (a plan is immutable after creation), and sk_flag_host on one
plan from several threads (serialised on the plan's staging buffers).  Every result
must equal the oracle's, whatever the interleaving."""

import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402
import synth  # noqa: E402
from oracle import digitisation as dg  # noqa: E402

pytestmark = pytest.mark.gpu


def _data(k, N, M, F):
    ds = synth.Dataset(n_frames=F, M=M, N=N, seed=synth.sub_seed(31, k),
                       rfi=synth.rfi_plan(synth.sub_seed(31, k), F, 0.1, 0.05))
    return ds.generate_cpu()


def _run_threads(fn, n):
    errors = []

    def wrap(k):
        try:
            fn(k)
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    th = [threading.Thread(target=wrap, args=(k,)) for k in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join(120)
    assert not any(t.is_alive() for t in th)
    if errors:
        raise errors[0]


def test_one_plan_many_streams():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda:0")
    N, M, F, n = 2048, 256, 40, 4
    xs = [_data(k, N, M, F) for k in range(n)]
    delta = -0.05
    wants = [oracle.flag(x, M, N, 3.0, delta) for x in xs]
    plan = sk.sk_plan_create(N, M, 3.0, delta)
    d_in = [torch.from_numpy(x.reshape(-1)).to(dev) for x in xs]
    outs = [(torch.full((F,), -1.0, dtype=torch.float32, device=dev),
             torch.full((F,), 7, dtype=torch.uint8, device=dev)) for _ in range(n)]
    torch.cuda.synchronize()

    def work(k):
        st = torch.cuda.Stream(dev)
        for _ in range(5):
            sk.sk_flag(plan, d_in[k], F, outs[k][0], outs[k][1], st)
        st.synchronize()

    try:
        _run_threads(work, n)
    finally:
        sk.sk_plan_destroy(plan)
    for w, (skv, mask) in zip(wants, outs):
        assert np.array_equal(mask.cpu().numpy(), w["mask"])
        assert np.array_equal(skv.cpu().numpy().view(np.uint32), w["sk"].view(np.uint32))


def test_flag_host_from_many_threads_on_one_plan():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    N, M, n = 512, 256, 4
    Fs = [300, 17, 129, 64]   # different sizes: chunk counts differ per call
    xs = [_data(10 + k, N, M, F) for k, F in enumerate(Fs)]
    ds0 = synth.Dataset(n_frames=1, M=M, N=N, seed=synth.sub_seed(31, 10))
    delta = float(np.mean(dg.delta_of_sigma(ds0.sigma)))
    wants = [oracle.flag(x, M, N, 3.0, delta) for x in xs]
    plan = sk.sk_plan_create(N, M, 3.0, delta)
    got = [None] * n

    def work(k):
        F = Fs[k]
        h_in = torch.from_numpy(xs[k].reshape(-1)).pin_memory()
        for _ in range(3):
            h_sk = torch.full((F,), -1.0, dtype=torch.float32).pin_memory()
            h_mask = torch.full((F,), 7, dtype=torch.uint8).pin_memory()
            sk.sk_flag_host(plan, h_in, F, h_sk, h_mask)
            r = (h_sk.numpy().copy(), h_mask.numpy().copy())
            if got[k] is not None:
                assert np.array_equal(r[1], got[k][1])
            got[k] = r

    try:
        _run_threads(work, n)
    finally:
        sk.sk_plan_destroy(plan)
    for w, (skv, mask) in zip(wants, got):
        assert np.array_equal(mask, w["mask"])
        assert np.array_equal(skv.view(np.uint32), w["sk"].view(np.uint32))
