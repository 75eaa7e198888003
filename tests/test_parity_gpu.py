"""Parity of the CUDA path with the oracle, through the C ABI.

Bar: S1, S2, Q, N_eff and masks bit-exact; SK fp32 bit-identical to the
oracle's kernel-precision statement and within 1e-6 relative of the fp64
oracle (Eq. final).  Inputs are seeded and synthetic (the `synth` generator,
or uniform random bytes that include nibble 0 = -8).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402
import synth  # noqa: E402
from oracle import digitisation as dg  # noqa: E402

pytestmark = pytest.mark.gpu

SK_REL = 1e-6


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda:0")


def run_compute(x, M, N, n_sigma=3.0, delta=0.0, layout=0, rows=None, grid=0):
    """sk_compute + sk_flag on bytes x [F, M*N]; numpy outputs."""
    dev = _dev()
    x = np.ascontiguousarray(x, dtype=np.uint8).reshape(-1, M * N)
    F = x.shape[0]
    d_in = torch.from_numpy(x.reshape(-1)).to(dev) if F else torch.empty(16, dtype=torch.uint8,
                                                                          device=dev)
    s1 = torch.full((max(F, 1), N), -1, dtype=torch.int32, device=dev)
    s2 = torch.full_like(s1, -1)
    q = torch.full((max(F, 1),), -1, dtype=torch.int64, device=dev)
    skv = torch.full((max(F, 1),), -1.0, dtype=torch.float32, device=dev)
    ne = torch.full((max(F, 1),), -1, dtype=torch.int32, device=dev)
    mask = torch.full((max(F, 1),), 7, dtype=torch.uint8, device=dev)
    sk2 = torch.full_like(skv, -1.0)
    plan = sk.sk_plan_create(N, M, n_sigma, delta, layout=layout)
    try:
        if rows is not None:
            sk.sk_plan_set_tiles(plan, rows, grid)
        sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
        sk.sk_flag(plan, d_in, F, sk2, mask)
        torch.cuda.synchronize()
        t_lo, t_hi = sk.sk_plan_thresholds(plan, N)
    finally:
        sk.sk_plan_destroy(plan)
    return dict(S1=s1.cpu().numpy()[:F], S2=s2.cpu().numpy()[:F], Q=q.cpu().numpy()[:F],
                neff=ne.cpu().numpy()[:F], sk=skv.cpu().numpy()[:F], sk_flag=sk2.cpu().numpy()[:F],
                mask=mask.cpu().numpy()[:F], t_lo=t_lo, t_hi=t_hi)


def assert_parity(got, want, check_sums=True):
    if check_sums:
        assert np.array_equal(got["S1"], want["S1"])
        assert np.array_equal(got["S2"], want["S2"])
    assert np.array_equal(got["Q"], want["Q"])
    assert np.array_equal(got["neff"], want["neff"])
    assert np.array_equal(got["sk"].view(np.uint32), want["sk"].view(np.uint32))
    assert np.array_equal(got["sk_flag"].view(np.uint32), want["sk"].view(np.uint32))
    assert np.array_equal(got["mask"], want["mask"])
    ok = np.isfinite(want["sk64"])
    rel = np.abs(got["sk"][ok] - want["sk64"][ok]) / np.maximum(np.abs(want["sk64"][ok]), 1e-30)
    near0 = np.abs(want["sk64"][ok]) < 1e-6
    assert np.all((rel <= SK_REL) | near0)
    assert np.all(np.isnan(got["sk"][~ok]))


def test_exact_conversions_match_cuda_intrinsics():
    """The epilogue's own int64 -> fp32 and fp32 -> int64 roundings (and the input
    term built on them) agree bit for bit with CUDA's conversion intrinsics: every
    non-negative fp32 below 2^62, every halfway case below 2^43 with its
    neighbours, and hashed samples."""
    _dev()
    n, bad = sk.sk_selftest_conversions(0)
    assert n == 0x5E800000 + (1 << 25) + 19 * (1 << 23) * 3 + (1 << 28) + (1 << 26) + (1 << 19)
    assert bad == 0


def test_pathfinder_workload_bit_exact():
    """N=256, M=256, 64 frames, CW frames 10-19, 50 % pulse frames 40-44, 3 sigma."""
    ds = synth.pathfinder_config()
    x = ds.generate_cpu()
    delta = float(np.mean(dg.delta_of_sigma(ds.sigma)))
    want = oracle.flag(x, 256, 256, 3.0, delta)
    got = run_compute(x, 256, 256, 3.0, delta)
    assert np.array_equal(got["t_lo"][1:], want["t_lo"][1:])
    assert np.array_equal(got["t_hi"][1:], want["t_hi"][1:])
    assert_parity(got, want)
    assert got["mask"][10:20].all()


def test_pathfinder_25pct_pulse_flags_high():
    ds = synth.pathfinder_config(duty=0.25)
    x = ds.generate_cpu()
    delta = float(np.mean(dg.delta_of_sigma(ds.sigma)))
    want = oracle.flag(x, 256, 256, 3.0, delta)
    got = run_compute(x, 256, 256, 3.0, delta)
    assert_parity(got, want)
    # above the digitisation-shifted centre 1 + delta (App. B), not necessarily above 1
    assert got["mask"][40:45].all() and (got["sk"][40:45] > 1.0 + delta).all()


@pytest.mark.parametrize("N,M,F", [
    (8, 16, 5), (16, 32, 33), (24, 48, 17), (256, 128, 40), (1000, 64, 9),
    (2048, 256, 7), (4096, 32, 5), (2048, 1024, 3), (512, 4096, 2), (64, 16, 70),
    (4096, 4096, 2), (768, 256, 7), (1040, 64, 9), (3008, 32, 5), (2056, 256, 5),
    (520, 32, 11)])
def test_fast_path_shapes_random_bytes(N, M, F):
    rng = np.random.default_rng(N * 7 + M + F)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    want = oracle.flag(x, M, N, 2.5, 0.0)
    for rows in (8, 16):
        got = run_compute(x, M, N, 2.5, 0.0, rows=rows)
        assert_parity(got, want)


@pytest.mark.parametrize("N,M,F,layout", [
    (1, 2, 3, 0), (3, 17, 4, 0), (100, 100, 6, 0), (257, 33, 5, 0), (4095, 16, 2, 0),
    (7, 64, 9, 0), (10, 6, 7, 0), (13, 3, 5, 0), (2046, 255, 2, 0), (4093, 7, 3, 0),
    (1, 2, 3, 1), (100, 100, 6, 1), (256, 256, 4, 1), (37, 5, 11, 1)])
def test_general_path_ragged_shapes(N, M, F, layout):
    rng = np.random.default_rng(N * 13 + M * 3 + F + layout)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    want = oracle.flag(x, M, N, 3.0, 0.1, layout=layout)
    got = run_compute(x, M, N, 3.0, 0.1, layout=layout)
    assert_parity(got, want)


def test_empty_single_and_dead_frames():
    M, N = 64, 128
    rng = np.random.default_rng(3)
    x = rng.integers(0, 256, size=(5, M, N), dtype=np.uint8)
    x[1, :, 7] = 0x88        # one dead input
    x[2] = 0x88              # no input has power
    x[3, :, :] = 0x00        # every sample (-8, -8): constant modulus, SK = 0
    x = x.reshape(5, -1)
    want = oracle.flag(x, M, N)
    got = run_compute(x, M, N)
    assert_parity(got, want)
    assert got["neff"][2] == 0 and got["mask"][2] == 1 and np.isnan(got["sk"][2])
    assert got["neff"][1] == N - 1 and got["Q"][3] == 0
    got1 = run_compute(x[:1], M, N)
    assert np.array_equal(got1["Q"], want["Q"][:1])
    got0 = run_compute(x[:0], M, N)
    assert got0["Q"].size == 0


def test_tiles_and_grid_do_not_change_results():
    rng = np.random.default_rng(17)
    M, N, F = 256, 2048, 37
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    ref = run_compute(x, M, N)
    for rows, grid in ((8, 0), (16, 1), (8, 5), (16, 300)):
        got = run_compute(x, M, N, rows=rows, grid=grid)
        for k in ("S1", "S2", "Q", "neff", "mask"):
            assert np.array_equal(got[k], ref[k])


def test_misaligned_and_bad_arguments_rejected():
    dev = _dev()
    buf = torch.zeros(4096 + 16, dtype=torch.uint8, device=dev)
    mask = torch.zeros(4, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(16, 16)
    try:
        with pytest.raises(sk.SkError) as e:
            sk.sk_flag(plan, buf.data_ptr() + 1, 1, None, mask)
        assert e.value.status == sk.SK_ERR_INVALID_ARG
        with pytest.raises(sk.SkError):
            sk.sk_flag(plan, buf, -1, None, mask)
        with pytest.raises(sk.SkError):
            sk.sk_flag(plan, buf, 1, None, None)
        with pytest.raises(sk.SkError):
            sk.sk_plan_set_tiles(plan, 12, 0)
    finally:
        sk.sk_plan_destroy(plan)


def test_gpu_generator_matches_cpu_generator():
    dev = _dev()
    ds = synth.full_array_config(n_freq=1, n_frames=40, N=512, M=128)[0]
    cpu = ds.generate_cpu()
    d = torch.empty(ds.nbytes, dtype=torch.uint8, device=dev)
    ds.generate_gpu(d)
    assert np.array_equal(d.cpu().numpy().reshape(cpu.shape), cpu)
    part = torch.empty(5 * ds.frame_bytes, dtype=torch.uint8, device=dev)
    ds.generate_gpu(part, frame0=11, n=5)
    assert np.array_equal(part.cpu().numpy().reshape(5, -1), cpu[11:16])


def test_flag_host_matches_device_path():
    dev = _dev()
    ds = synth.full_array_config(n_freq=1, n_frames=300, N=512, M=256)[0]
    x = ds.generate_cpu()
    delta = float(np.mean(dg.delta_of_sigma(ds.sigma)))
    want = oracle.flag(x, 256, 512, 3.0, delta)
    h_in = torch.from_numpy(x.reshape(-1)).pin_memory()
    h_sk = torch.zeros(300, dtype=torch.float32).pin_memory()
    h_mask = torch.zeros(300, dtype=torch.uint8).pin_memory()
    plan = sk.sk_plan_create(512, 256, 3.0, delta)
    try:
        sk.sk_flag_host(plan, h_in, 300, h_sk, h_mask)
    finally:
        sk.sk_plan_destroy(plan)
    assert np.array_equal(h_mask.numpy(), want["mask"])
    assert np.array_equal(h_sk.numpy().view(np.uint32), want["sk"].view(np.uint32))


def _full_size_every_frame(datasets, n_sigma=3.0):
    """Run sk_compute (S1, S2, Q, SK, N_eff) and sk_flag (SK, mask) on a whole
    multi-frequency workload in one launch each -- the launch shape the benchmark
    times, row-balanced over the grid -- and compare EVERY frame with the oracle.
    The bytes come from the CPU generator and are uploaded, so the oracle's input
    never passes through CUDA code; the oracle runs per frequency on the same bytes."""
    dev = _dev()
    ds0 = datasets[0]
    M, N, layout = ds0.M, ds0.N, ds0.layout
    F = sum(d.n_frames for d in datasets)
    d_in = torch.empty(F * M * N, dtype=torch.uint8, device=dev)
    host = []
    off = 0
    for d in datasets:
        x = d.generate_cpu()
        d_in[off:off + d.nbytes].copy_(torch.from_numpy(x.reshape(-1)))
        host.append(x)
        off += d.nbytes
    sigma = np.concatenate([d.sigma for d in datasets])
    delta = float(np.mean(dg.delta_of_sigma(sigma)))
    s1 = torch.empty((F, N), dtype=torch.int32, device=dev)
    s2 = torch.empty_like(s1)
    q = torch.empty(F, dtype=torch.int64, device=dev)
    skv = torch.empty(F, dtype=torch.float32, device=dev)
    ne = torch.empty(F, dtype=torch.int32, device=dev)
    mask = torch.empty(F, dtype=torch.uint8, device=dev)
    sk2 = torch.empty(F, dtype=torch.float32, device=dev)
    plan = sk.sk_plan_create(N, M, n_sigma, delta, layout=layout)
    try:
        sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
        sk.sk_flag(plan, d_in, F, sk2, mask)
        torch.cuda.synchronize()
    finally:
        sk.sk_plan_destroy(plan)
    del d_in
    torch.cuda.empty_cache()
    s1, s2, q, skv, ne, mask, sk2 = (t.cpu().numpy() for t in (s1, s2, q, skv, ne, mask, sk2))
    rel = []
    f0 = 0
    for d, x in zip(datasets, host):
        w = oracle.flag(x, M, N, n_sigma, delta, layout=layout)
        sl = slice(f0, f0 + d.n_frames)
        assert np.array_equal(s1[sl], w["S1"]) and np.array_equal(s2[sl], w["S2"])
        assert np.array_equal(q[sl], w["Q"]) and np.array_equal(ne[sl], w["neff"])
        assert np.array_equal(skv[sl].view(np.uint32), w["sk"].view(np.uint32))
        assert np.array_equal(sk2[sl].view(np.uint32), w["sk"].view(np.uint32))
        assert np.array_equal(mask[sl], w["mask"])
        rel.append(np.abs(skv[sl].astype(np.float64) - w["sk64"]) / np.abs(w["sk64"]))
        f0 += d.n_frames
    rel = np.concatenate(rel)
    assert rel.max() <= SK_REL
    print(f"every frame checked: {F} frames, {F * M * N / 1e9:.2f} GB, layout {layout}, "
          f"flagged {int(mask.sum())}, SK fp32 vs fp64 max rel {rel.max():.3g} "
          f"mean {rel.mean():.3g}")
    return dict(mask=mask, F=F, checked=F)


def test_full_array_workload_every_frame():
    """4 frequencies x N=2048, M=256, 1525 frames (3.2 GB, the benchmark launch):
    S1, S2, Q, N_eff, SK bits and masks of all 6100 frames against the oracle."""
    datasets = synth.full_array_config()
    r = _full_size_every_frame(datasets)
    assert r["checked"] == 4 * 1525
    # the strong CW frames are flagged; clean frames mostly are not
    cw = [1525 * k + x.frame for k, d in enumerate(datasets) for x in d.rfi if x.kind == "cw"
          and x.amp > 2.5]
    assert r["mask"][cw].all()
    assert r["mask"].mean() < 0.06


@pytest.mark.parametrize("N,M,layout,F", [
    (2047, 256, 0, 23), (100, 100, 0, 301), (2056, 256, 0, 19), (520, 256, 0, 77),
    (2048, 48, 0, 61), (2048, 100, 0, 41), (2048, 64, 1, 45), (2048, 4096, 1, 3)])
def test_benchmarked_off_shapes_bit_exact(N, M, layout, F):
    """The shapes the benchmark times besides its own (ragged N, N = 8 mod 16, a short
    integration, input-major M = 64 and 4096), each over several CTAs' worth of
    frames with a ragged tail: everything bit-exact against the oracle."""
    rng = np.random.default_rng(N * 11 + M * 3 + layout)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    want = oracle.flag(x, M, N, 3.0, 0.0, layout=layout)
    got = run_compute(x, M, N, 3.0, 0.0, layout=layout)
    assert_parity(got, want)


@pytest.mark.parametrize("N,M,F", [
    (2048, 100, 61),    # 7 turns of 16 rows, the last with 4
    (256, 100, 201),    # one-warp teams
    (1000, 50, 77),     # N = 8 mod 16, a partial last slice
    (4096, 24, 33),     # 16-warp teams, one per CTA
    (512, 2, 999),      # the shortest integration: one turn of 2 rows
    (2056, 17, 40),     # 9-warp teams (no folded tail with a partial turn)
    (768, 200, 19),     # 13 turns, the last with 8 rows
    (264, 7, 301),
])
def test_partial_last_turn_bit_exact(N, M, F):
    """Time-major N a multiple of 8 (256..4096) with M not a multiple of 16: whole-
    frame warp slices whose last 16-row turn is partial (rows past M read nothing);
    the team path asked for instead takes the general path.  S1, S2, Q, N_eff, SK
    bits, masks and the per-input estimates against the oracle."""
    dev = _dev()
    rng = np.random.default_rng(N * 5 + M + F)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    x[F // 2, : 3 * N] = 0x88                 # dead rows at the start of a frame
    want = oracle.flag(x, M, N, 3.0, 0.05)
    got = run_compute(x, M, N, 3.0, 0.05)
    assert_parity(got, want)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    wi = oracle.flag_inputs(x, M, N, 3.0, 0.05)
    for path, taken in ((sk.SK_PATH_AUTO, sk.SK_PATH_WARP_SLICE),
                        (sk.SK_PATH_TEAM, sk.SK_PATH_GENERAL)):
        plan = sk.sk_plan_create(N, M, 3.0, 0.05)
        try:
            sk.sk_plan_set_config(plan, rows=8, path=path)
            sk_in = torch.empty((F, N), dtype=torch.float32, device=dev)
            m_in = torch.empty((F, N), dtype=torch.uint8, device=dev)
            mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
            sk.sk_compute_inputs(plan, d_in, F, sk_in, m_in)
            sk.sk_flag(plan, d_in, F, None, mask)
            torch.cuda.synchronize()
            assert sk.sk_plan_get_config(plan)["last_path"] == taken
        finally:
            sk.sk_plan_destroy(plan)
        assert np.array_equal(sk_in.cpu().numpy().view(np.uint32), wi["sk_in"].view(np.uint32))
        assert np.array_equal(m_in.cpu().numpy(), wi["mask_in"])
        assert np.array_equal(mask.cpu().numpy(), want["mask"])


@pytest.mark.parametrize("N,M,F", [(256, 256, 40), (2048, 128, 6), (100, 64, 9)])
def test_independent_estimates_bit_exact(N, M, F):
    """sk_compute_inputs: per-input SK^_i and one-input flags against the oracle."""
    dev = _dev()
    rng = np.random.default_rng(N + M + F)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    x[1, ::N] = 0x88
    want = oracle.flag_inputs(x, M, N, 3.0, 0.05)
    whole = oracle.flag(x, M, N, 3.0, 0.05)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    sk_in = torch.empty((F, N), dtype=torch.float32, device=dev)
    m_in = torch.empty((F, N), dtype=torch.uint8, device=dev)
    skv = torch.empty(F, dtype=torch.float32, device=dev)
    mask = torch.empty(F, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N, M, 3.0, 0.05)
    try:
        sk.sk_compute_inputs(plan, d_in, F, sk_in, m_in, skv, mask)
        torch.cuda.synchronize()
    finally:
        sk.sk_plan_destroy(plan)
    got = sk_in.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want["sk_in"].view(np.uint32))
    assert np.array_equal(m_in.cpu().numpy(), want["mask_in"])
    assert np.array_equal(mask.cpu().numpy(), whole["mask"])
    ok = want["valid"] == 1
    rel = np.abs(got[ok] - want["sk_in64"][ok]) / np.maximum(np.abs(want["sk_in64"][ok]), 1e-6)
    assert rel.max() <= SK_REL


@pytest.mark.parametrize("N,M", [(256, 64), (16, 32), (2048, 256)])
def test_pearson3_thresholds_and_masks_bit_exact(N, M):
    """SK_THRESH_PEARSON3: plan thresholds and masks equal the oracle's."""
    dev = _dev()
    ds = synth.Dataset(n_frames=80, M=M, N=N, seed=synth.sub_seed(7, N + M),
                       rfi=synth.rfi_plan(synth.sub_seed(7, N + M), 80, 0.1, 0.05))
    x = ds.generate_cpu()
    delta = float(np.mean(dg.delta_of_sigma(ds.sigma)))
    want = oracle.flag(x, M, N, 2.0, delta, pearson3=True)
    plan = sk.sk_plan_create(N, M, 2.0, delta, flags=sk.SK_THRESH_PEARSON3)
    try:
        t_lo, t_hi = sk.sk_plan_thresholds(plan, N)
        d_in = torch.from_numpy(x.reshape(-1)).to(dev)
        mask = torch.empty(80, dtype=torch.uint8, device=dev)
        sk.sk_flag(plan, d_in, 80, None, mask)
        torch.cuda.synchronize()
    finally:
        sk.sk_plan_destroy(plan)
    assert np.array_equal(t_lo[1:], want["t_lo"][1:]) and np.array_equal(t_hi[1:], want["t_hi"][1:])
    assert np.array_equal(mask.cpu().numpy(), want["mask"])


@pytest.mark.parametrize("N,M,F", [(2048, 256, 9), (256, 256, 37), (100, 128, 11), (7, 1024, 5),
                                   (1, 128, 3), (512, 2048, 3), (4096, 128, 2), (33, 384, 6),
                                   (2048, 64, 21), (33, 64, 9), (4096, 64, 5), (3, 64, 40)])
def test_input_major_fast_path_bit_exact(N, M, F):
    """Layout [frame][input][t] through the input-major paths: grouped for M = 64 and
    128 * 2^k (with sub-inputs above 512), per-input for other multiples of 16 G."""
    rng = np.random.default_rng(N * 3 + M * 5 + F)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    x[0, : M] = 0x88                       # input 0 of frame 0 has no power
    want = oracle.flag(x, M, N, 3.0, 0.05, layout=1)
    got = run_compute(x, M, N, 3.0, 0.05, layout=1)
    assert_parity(got, want)
    # independent estimates through the same path
    dev = _dev()
    wi = oracle.flag_inputs(x, M, N, 3.0, 0.05, layout=1)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    sk_in = torch.empty((F, N), dtype=torch.float32, device=dev)
    m_in = torch.empty((F, N), dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N, M, 3.0, 0.05, layout=1)
    try:
        sk.sk_compute_inputs(plan, d_in, F, sk_in, m_in)
        torch.cuda.synchronize()
    finally:
        sk.sk_plan_destroy(plan)
    assert np.array_equal(sk_in.cpu().numpy().view(np.uint32), wi["sk_in"].view(np.uint32))
    assert np.array_equal(m_in.cpu().numpy(), wi["mask_in"])


def test_full_array_input_major_every_frame():
    """The same 3.2 GB workload in the input-major layout [frame][input][t] (the
    row-balanced grouped input-major launch the benchmark times): every frame
    against the oracle."""
    import dataclasses

    datasets = [dataclasses.replace(d, layout=1) for d in synth.full_array_config()]
    r = _full_size_every_frame(datasets)
    assert r["checked"] == 4 * 1525


@pytest.mark.parametrize("N,M,F", [(4096, 1024, 2), (4096, 4096, 1), (9, 512, 4), (33, 2048, 3),
                                   (5, 4096, 2), (1000, 1024, 3)])
def test_input_major_maximum_and_ragged_sizes(N, M, F):
    """Input-major at the largest N and M (the grouped path reads inputs longer than 512
    samples as 2, 4 or 8 sub-inputs) and ragged N; worst-case bytes (every sample
    -8-8j) in one frame."""
    rng = np.random.default_rng(N + M + F)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    x[F - 1, : M * min(N, 64)] = 0x00
    want = oracle.flag(x, M, N, 3.0, 0.0, layout=1)
    got = run_compute(x, M, N, 3.0, 0.0, layout=1)
    assert_parity(got, want)


def test_random_shapes_sweep():
    """40 seeded random shapes (N, M, frames, layout) across every path: vector and
    general time-major, grouped (with sub-inputs), per-input and general input-major.
    Random bytes, nibble 0 included; everything bit-exact against the oracle."""
    rng = np.random.default_rng(20261204)
    Ms = [2, 3, 16, 32, 48, 64, 100, 128, 256, 384, 512, 1024, 2048, 4096]
    for case in range(40):
        layout = int(rng.integers(0, 2))
        M = int(rng.choice(Ms)) if rng.random() < 0.7 else int(rng.integers(2, 700))
        N = int(rng.integers(1, 4097)) if rng.random() < 0.5 else int(8 * rng.integers(1, 513))
        F = int(rng.integers(1, 7))
        while F > 1 and F * M * N > (6 << 20):
            F -= 1
        if M * N > (16 << 20):
            N = max(1, (16 << 20) // M)
        x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
        want = oracle.flag(x, M, N, 2.5, -0.02, layout=layout)
        got = run_compute(x, M, N, 2.5, -0.02, layout=layout)
        try:
            assert_parity(got, want)
        except AssertionError as e:
            raise AssertionError(f"case {case}: N={N} M={M} F={F} layout={layout}") from e
