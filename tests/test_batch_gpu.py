"""Batched persistent launch (many frequencies of different N and M in one
graph-captured launch) against the oracle and the plain launch."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402
import synth  # noqa: E402
from oracle import digitisation as dg  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda:0")


@pytest.mark.parametrize("shapes", [
    # every kernel class: N = 2048 (16- and 8-row tiles), N = 256, other N on the
    # fast path, the general path, input-major items, empty items
    [(2048, 256, 23, 0), (256, 128, 70, 0), (2048, 1024, 5, 0), (256, 1024, 31, 0),
     (100, 48, 9, 0), (512, 256, 1, 0), (2048, 128, 0, 0), (256, 256, 64, 0),
     (2048, 48, 4, 0), (256, 256, 10, 1), (2048, 128, 3, 1)],
    # input-major items only: the grouped path per M, ragged N, and the general path
    [(2048, 256, 9, 1), (256, 1024, 7, 1), (512, 512, 5, 1), (100, 128, 6, 1), (64, 64, 4, 1),
     (2048, 128, 11, 1), (2048, 64, 37, 1), (33, 64, 6, 1)],
    # time-major N = 2048 items of M <= 128 (the warp-slice class, one item long
    # enough that each team's slot ring wraps), beside N = 2048 items of larger M
    [(2048, 128, 19, 0), (2048, 64, 33, 0), (2048, 32, 3000, 0), (2048, 96, 7, 0),
     (2048, 256, 5, 0), (2048, 128, 1, 0), (2048, 1024, 2, 0)],
    # one class only
    [(256, 256, 40, 0), (256, 128, 17, 0)],
    [(2048, 256, 7, 0)],
    # nothing to do
    [(2048, 256, 0, 0), (256, 128, 0, 0)]])
def test_mixed_batch_matches_oracle_and_replays(shapes):
    dev = _dev()
    items, plans, bufs, wants = [], [], [], []
    for k, (N, M, F, layout) in enumerate(shapes):
        ds = synth.Dataset(n_frames=max(F, 1), M=M, N=N, seed=synth.sub_seed(2, k), layout=layout,
                           rfi=synth.rfi_plan(synth.sub_seed(2, k), max(F, 1), 0.2, 0.1))
        x = ds.generate_cpu()[:F]
        delta = float(np.mean(dg.delta_of_sigma(ds.sigma)))
        wants.append(oracle.flag(x, M, N, 3.0, delta, layout=layout) if F else None)
        plan = sk.sk_plan_create(N, M, 3.0, delta, layout=layout)
        d_in = torch.from_numpy(x.reshape(-1)).to(dev) if F else torch.empty(16, dtype=torch.uint8,
                                                                             device=dev)
        skv = torch.full((max(F, 1),), -1.0, dtype=torch.float32, device=dev)
        mask = torch.full((max(F, 1),), 9, dtype=torch.uint8, device=dev)
        plans.append(plan)
        bufs.append((d_in, skv, mask))
        items.append((plan, d_in, F, skv, mask))
    batch = sk.sk_batch_create(items)
    try:
        for rep in range(2):
            for _, skv, mask in bufs:
                skv.fill_(-1.0)
                mask.fill_(9)
            sk.sk_batch_run(batch)
            torch.cuda.synchronize()
            for (N, M, F, _), w, (_, skv, mask) in zip(shapes, wants, bufs):
                if F == 0:
                    assert mask[0].item() == 9
                    continue
                assert np.array_equal(mask.cpu().numpy()[:F], w["mask"])
                assert np.array_equal(skv.cpu().numpy()[:F].view(np.uint32),
                                      w["sk"].view(np.uint32))
    finally:
        sk.sk_batch_destroy(batch)
        for p in plans:
            sk.sk_plan_destroy(p)


def test_batch_rejects_bad_items():
    dev = _dev()
    plan = sk.sk_plan_create(256, 256)
    buf = torch.zeros(256 * 256 + 16, dtype=torch.uint8, device=dev)
    mask = torch.zeros(1, dtype=torch.uint8, device=dev)
    try:
        with pytest.raises(sk.SkError):
            sk.sk_batch_create([(plan, buf.data_ptr() + 8, 1, None, mask)])
        with pytest.raises(sk.SkError):
            sk.sk_batch_create([(plan, buf, 1, None, None)])
        with pytest.raises(sk.SkError):
            sk.sk_batch_create([])
    finally:
        sk.sk_plan_destroy(plan)


def test_randomised_batches_against_the_oracle():
    """Three seeded random batches of 12 items each: N, M, frame counts and layouts
    drawn at random (every kernel class appears), replayed twice; every item equals
    the oracle."""
    dev = _dev()
    rng = np.random.default_rng(404)
    Ns = [8, 37, 100, 256, 512, 1000, 2048, 4096]
    Ms = [16, 48, 64, 100, 128, 256, 512, 1024, 2048]
    for rep in range(3):
        items, plans, bufs, wants = [], [], [], []
        for k in range(12):
            N, M = int(rng.choice(Ns)), int(rng.choice(Ms))
            layout = int(rng.integers(0, 2))
            F = int(rng.integers(0, 9))
            while F > 1 and F * M * N > (8 << 20):
                F -= 1
            x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
            delta = float(rng.uniform(-0.1, 0.0))
            wants.append(oracle.flag(x, M, N, 3.0, delta, layout=layout) if F else None)
            plan = sk.sk_plan_create(N, M, 3.0, delta, layout=layout)
            d_in = (torch.from_numpy(x.reshape(-1)).to(dev) if F
                    else torch.empty(16, dtype=torch.uint8, device=dev))
            skv = torch.full((max(F, 1),), -1.0, dtype=torch.float32, device=dev)
            mask = torch.full((max(F, 1),), 9, dtype=torch.uint8, device=dev)
            plans.append(plan)
            bufs.append((F, skv, mask))
            items.append((plan, d_in, F, skv, mask))
        batch = sk.sk_batch_create(items)
        try:
            for _ in range(2):
                sk.sk_batch_run(batch)
                torch.cuda.synchronize()
                for k, ((F, skv, mask), w) in enumerate(zip(bufs, wants)):
                    if not F:
                        continue
                    assert np.array_equal(mask.cpu().numpy()[:F], w["mask"]), (rep, k)
                    assert np.array_equal(skv.cpu().numpy()[:F].view(np.uint32),
                                          w["sk"].view(np.uint32)), (rep, k)
        finally:
            sk.sk_batch_destroy(batch)
            for p in plans:
                sk.sk_plan_destroy(p)
