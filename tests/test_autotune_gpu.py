"""The autotuner's launch configurations: a cache entry read by sk_plan_create (and
by sk_batch_create through the plan) changes the path the launch takes, and the
results stay bit-exact against the oracle under every configuration; a short
tuning sweep writes a cache that plans then read back."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402
from paper_1808_10365_b300 import autotune  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda:0")


def _flag(plan, x, F, dev):
    d_in = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(dev)
    skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
    mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
    sk.sk_flag(plan, d_in, F, skv, mask)
    torch.cuda.synchronize()
    return skv.cpu().numpy(), mask.cpu().numpy()


def _exact(got, want):
    assert np.array_equal(got[1], want["mask"])
    assert np.array_equal(got[0].view(np.uint32), want["sk"].view(np.uint32))


@pytest.mark.parametrize("N,M,layout,entry,taken", [
    (2048, 256, 0, None, sk.SK_PATH_ROW_BALANCED),
    (2048, 256, 0, "16 0 1 0 0 0", sk.SK_PATH_TEAM),
    (2048, 256, 0, "16 0 2 0 1 0", sk.SK_PATH_WARP_SLICE),
    (2048, 256, 0, "8 0 0 0 0 0", sk.SK_PATH_TEAM),
    (1000, 128, 0, "16 0 1 0 0 0", sk.SK_PATH_TEAM),
    (2048, 256, 1, None, sk.SK_PATH_ROW_BALANCED),
    (2048, 256, 1, "16 0 1 7 1 0", sk.SK_PATH_TEAM),
    (2048, 256, 1, "16 0 2 8 0 0", sk.SK_PATH_WARP_SLICE),
    (256, 96, 1, "16 0 0 6 0 0", sk.SK_PATH_PER_INPUT),
    (2048, 64, 1, "16 0 3 6 1 0", sk.SK_PATH_ROW_BALANCED),
    (2048, 48, 0, "8 0 1 0 0 0", sk.SK_PATH_TEAM),
    (2048, 48, 0, None, sk.SK_PATH_ROW_BALANCED),
    (2047, 256, 0, None, sk.SK_PATH_ROW_BALANCED),
    (2047, 256, 0, "16 0 1 0 0 0", sk.SK_PATH_GENERAL),
    (100, 100, 0, None, sk.SK_PATH_STREAM),
    (100, 100, 0, "8 0 1 0 0 0", sk.SK_PATH_GENERAL),
    (128, 256, 0, "16 0 6 0 0 0", sk.SK_PATH_STREAM),
    (128, 256, 0, None, sk.SK_PATH_TEAM),
])
def test_cache_entry_sets_the_path_and_results_stay_exact(tmp_path, monkeypatch, N, M, layout,
                                                          entry, taken):
    dev = _dev()
    cache = tmp_path / "tiles.txt"
    cache.write_text("# test\n" + (f"{N} {M} {layout} {entry}\n" if entry else ""))
    monkeypatch.setenv("SK_AUTOTUNE_CACHE", str(cache))
    F = max(9, (48 << 20) // (N * M))
    rng = np.random.default_rng(N + M + layout)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    want = oracle.flag(x, M, N, 3.0, 0.0, layout=layout)
    plan = sk.sk_plan_create(N, M, 3.0, 0.0, layout=layout)
    try:
        cfg = sk.sk_plan_get_config(plan)
        if entry:
            rows, grid, path, team, pf, bp = (int(v) for v in entry.split())
            assert (cfg["rows"], cfg["grid_ctas"], cfg["path"], cfg["prefetch"],
                    cfg["batch_path"]) == (rows, grid, path, pf, bp)
            if team:
                assert cfg["team_log2"] == team
        assert cfg["last_path"] == 0
        _exact(_flag(plan, x, F, dev), want)
        assert sk.sk_plan_get_config(plan)["last_path"] == taken
    finally:
        sk.sk_plan_destroy(plan)


def test_set_config_rejects_bad_values():
    _dev()
    plan = sk.sk_plan_create(2048, 256, 3.0, 0.0)
    try:
        for bad in (dict(rows=12), dict(path=4), dict(batch_path=-1), dict(prefetch=2),
                    dict(team_log2=6)):       # team size: input-major plans only
            with pytest.raises(sk.SkError) as e:
                sk.sk_plan_set_config(plan, **bad)
            assert e.value.status == sk.SK_ERR_INVALID_ARG
    finally:
        sk.sk_plan_destroy(plan)


def test_batch_path_from_the_cache(tmp_path, monkeypatch):
    """Items of time-major N = 2048: by default M = 128 takes the warp-slice class and
    M = 256 the team class (two launches a run); a cache entry asking for warp slices
    at M = 256, or for the team path at M = 128, puts both in one class (one launch);
    masks exact either way."""
    dev = _dev()
    rng = np.random.default_rng(77)
    shapes = [(2048, 128, 23), (2048, 256, 17)]
    xs = [rng.integers(0, 256, size=(F, M * N), dtype=np.uint8) for N, M, F in shapes]
    wants = [oracle.flag(x, M, N, 3.0, 0.0) for x, (N, M, F) in zip(xs, shapes)]
    d_in = [torch.from_numpy(x.reshape(-1)).to(dev) for x in xs]
    for entry, launches in ((None, 2), ("2048 256 0 16 0 0 0 0 2", 1),
                            ("2048 128 0 16 0 0 0 0 1", 1)):
        cache = tmp_path / "tiles.txt"
        cache.write_text((entry + "\n") if entry else "")
        monkeypatch.setenv("SK_AUTOTUNE_CACHE", str(cache))
        plans = [sk.sk_plan_create(N, M, 3.0, 0.0) for N, M, F in shapes]
        outs = [(torch.full((F,), -1.0, dtype=torch.float32, device=dev),
                 torch.full((F,), 7, dtype=torch.uint8, device=dev)) for N, M, F in shapes]
        batch = sk.sk_batch_create([(p, d, F, s, m) for p, d, (N, M, F), (s, m)
                                    in zip(plans, d_in, shapes, outs)], 0)
        try:
            assert sk.sk_batch_launches(batch) == launches
            sk.sk_batch_run(batch)
            torch.cuda.synchronize()
            for (s, m), w in zip(outs, wants):
                _exact((s.cpu().numpy(), m.cpu().numpy()), w)
        finally:
            sk.sk_batch_destroy(batch)
            for p in plans:
                sk.sk_plan_destroy(p)


def test_sweep_writes_a_cache_the_plans_read(tmp_path, monkeypatch):
    """A short sweep (64 MB per shape) over both layouts: every configuration it
    timed took a valid path, its winner goes to the cache, and plans made with
    that cache carry the winner's configuration."""
    _dev()
    monkeypatch.setenv("SK_AUTOTUNE_CACHE", str(tmp_path / "none.txt"))
    entries = [autotune.tune(512, 256, 0, bytes_target=64 << 20, reps=2, rounds=1),
               autotune.tune(512, 256, 1, bytes_target=64 << 20, reps=2, rounds=1)]
    for e in entries:
        assert len(e["table"]) >= 4
        assert all(t["taken"] in ("team", "warp-slice", "row-balanced") for t in e["table"])
    out = tmp_path / "tiles.txt"
    autotune.write_cache(str(out), entries)
    monkeypatch.setenv("SK_AUTOTUNE_CACHE", str(out))
    for e in entries:
        plan = sk.sk_plan_create(512, 256, 3.0, 0.0, layout=e["layout"])
        try:
            cfg = sk.sk_plan_get_config(plan)
            for k in ("rows", "grid_ctas", "path", "prefetch", "batch_path"):
                assert cfg[k] == e[k]
            if e["team_log2"]:
                assert cfg["team_log2"] == e["team_log2"]
        finally:
            sk.sk_plan_destroy(plan)


def test_sustained_sweep(tmp_path, monkeypatch):
    """The sustained mode (each configuration streamed back to back, in order and in
    reverse) times every configuration, keeps the default unless another wins, and
    writes a cache line the plans read back."""
    _dev()
    monkeypatch.setenv("SK_AUTOTUNE_CACHE", str(tmp_path / "none.txt"))
    e = autotune.tune(512, 256, 0, bytes_target=64 << 20, sustained_s=0.05)
    assert e["sustained_s"] == 0.05 and len(e["table"]) >= 4
    assert all(t["ms"] > 0 and t["taken"] in ("team", "warp-slice", "row-balanced")
               for t in e["table"])
    assert "batch_table" not in e
    out = tmp_path / "tiles.txt"
    autotune.write_cache(str(out), [e])
    monkeypatch.setenv("SK_AUTOTUNE_CACHE", str(out))
    plan = sk.sk_plan_create(512, 256, 3.0, 0.0)
    try:
        cfg = sk.sk_plan_get_config(plan)
        assert (cfg["rows"], cfg["path"], cfg["prefetch"]) == (e["rows"], e["path"], e["prefetch"])
    finally:
        sk.sk_plan_destroy(plan)


def test_random_configurations_stay_exact():
    """40 seeded random shapes (both layouts, ragged N, M of any multiple of 16 and
    others) each under a random launch configuration (path, tile rows, grid, team
    size, prefetch): S1, S2, Q, N_eff, SK bits and masks bit-exact against the
    oracle, whatever path the configuration leads to."""
    dev = _dev()
    rng = np.random.default_rng(1808_2)
    taken = set()
    for case in range(40):
        layout = int(rng.integers(0, 2))
        N = int(rng.choice([int(rng.integers(1, 4097)), int(8 * rng.integers(1, 513))]))
        M = int(rng.choice([16, 32, 48, 64, 96, 128, 256, 512, 1024, 2048, 4096, 100, 2]))
        F = int(rng.integers(1, 300))
        while F > 1 and F * M * N > (12 << 20):
            F //= 2
        x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
        want = oracle.flag(x, M, N, 3.0, 0.01, layout=layout)
        plan = sk.sk_plan_create(N, M, 3.0, 0.01, layout=layout)
        try:
            team0 = sk.sk_plan_get_config(plan)["team_log2"]
            cfg = dict(rows=int(rng.choice([8, 16])), grid_ctas=int(rng.choice([0, 0, 37, 300])),
                       path=int(rng.integers(0, 4)), prefetch=int(rng.integers(0, 2)))
            if team0 and rng.random() < 0.5:
                cfg["team_log2"] = int(min(8 if team0 <= 8 else 9, max(5, team0 + rng.integers(-1, 2))))
            sk.sk_plan_set_config(plan, **cfg)
            d_in = torch.from_numpy(x.reshape(-1)).to(dev)
            s1 = torch.full((F, N), -1, dtype=torch.int32, device=dev)
            s2 = torch.full_like(s1, -1)
            q = torch.full((F,), -1, dtype=torch.int64, device=dev)
            skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
            ne = torch.full((F,), -1, dtype=torch.int32, device=dev)
            mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
            sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
            sk.sk_flag(plan, d_in, F, None, mask)
            torch.cuda.synchronize()
            taken.add(sk.sk_plan_get_config(plan)["last_path"])
        finally:
            sk.sk_plan_destroy(plan)
        tag = f"case {case}: N={N} M={M} F={F} layout={layout} cfg={cfg}"
        assert np.array_equal(s1.cpu().numpy(), want["S1"]), tag
        assert np.array_equal(s2.cpu().numpy(), want["S2"]), tag
        assert np.array_equal(q.cpu().numpy(), want["Q"]), tag
        assert np.array_equal(ne.cpu().numpy(), want["neff"]), tag
        assert np.array_equal(skv.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32)), tag
        assert np.array_equal(mask.cpu().numpy(), want["mask"]), tag
    assert len(taken) >= 4, taken
