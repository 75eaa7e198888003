"""Parity of the stream path (time-major frames of few inputs, SK_PATH_STREAM) with
the oracle, through the C ABI.

The stream path reads each frame as one run of 16-byte chunks.  Frames whose size
M N is not a multiple of 16 start at every offset from a 16-byte boundary, so their
first and last chunks hold bytes of the neighbouring frames (or lie partly outside
the input at its two ends); units of s lanes with 16 s a multiple of N keep each
chunk byte on one input.  Bar: S1, S2, Q, N_eff, masks and the fp32 SK bit-exact
(Eq. 1, Eq. singlesums, Eq. final, Sec. 3.2 test), per-input SK^_i too.
"""

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


def run_stream(x, M, N, n_sigma=2.5, delta=-0.01, grid=0, path=sk.SK_PATH_STREAM):
    dev = _dev()
    x = np.ascontiguousarray(x, dtype=np.uint8).reshape(-1, M * N)
    F = x.shape[0]
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    s1 = torch.full((F, N), -1, dtype=torch.int32, device=dev)
    s2 = torch.full_like(s1, -1)
    q = torch.full((F,), -1, dtype=torch.int64, device=dev)
    skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
    ne = torch.full((F,), -1, dtype=torch.int32, device=dev)
    sk2 = torch.full_like(skv, -1.0)
    mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N, M, n_sigma, delta)
    try:
        sk.sk_plan_set_config(plan, rows=16 if M % 32 == 0 else 8, grid_ctas=grid, path=path)
        sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
        sk.sk_flag(plan, d_in, F, sk2, mask)
        torch.cuda.synchronize()
        taken = sk.sk_plan_get_config(plan)["last_path"]
    finally:
        sk.sk_plan_destroy(plan)
    return taken, dict(S1=s1.cpu().numpy(), S2=s2.cpu().numpy(), Q=q.cpu().numpy(),
                       neff=ne.cpu().numpy(), sk=skv.cpu().numpy(), sk_flag=sk2.cpu().numpy(),
                       mask=mask.cpu().numpy())


def check(got, want, label):
    for k in ("S1", "S2", "Q", "neff", "mask"):
        assert np.array_equal(got[k], want[k]), f"{label}: {k}"
    assert np.array_equal(got["sk"].view(np.uint32), want["sk"].view(np.uint32)), label
    assert np.array_equal(got["sk_flag"].view(np.uint32), want["sk"].view(np.uint32)), label


# (N, M, F, grid): units inside one warp (N / gcd(N, 16) <= 32) and teams of several
# warps; frames of a multiple of 16 bytes and frames at every offset from a 16-byte
# boundary (M N odd); one round per CTA and many (small grids); frames smaller than
# one pass of a unit.
SHAPES = [
    (100, 100, 37, 0), (100, 100, 200, 3), (99, 101, 23, 0), (99, 101, 90, 2),
    (8, 256, 300, 0), (8, 256, 700, 5), (16, 64, 129, 0), (24, 256, 61, 0), (48, 256, 40, 4),
    (64, 100, 50, 0), (96, 256, 19, 0), (120, 100, 33, 0), (127, 3, 401, 0), (200, 100, 25, 2),
    (250, 200, 9, 0), (255, 17, 77, 1), (1, 2, 1000, 0), (1, 4096, 7, 0), (3, 17, 333, 0),
    (5, 1000, 12, 0), (7, 3, 999, 0), (12, 33, 257, 2), (33, 64, 64, 0), (300, 64, 20, 0),
    (500, 48, 11, 0), (512, 7, 31, 0), (1000, 16, 6, 0), (2, 2, 4097, 1),
]


@pytest.mark.parametrize("N,M,F,grid", SHAPES)
def test_stream_path_bit_exact(N, M, F, grid):
    """Random bytes (nibble 0 included) on the stream path against the oracle."""
    rng = np.random.default_rng(N * 7919 + M * 31 + F)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    if F > 3:
        x[1] = 0x88             # a frame without power: N_eff = 0, SK NaN, mask 1
        x[2, ::N] = 0x88        # input 0 without power in one frame
    want = oracle.flag(x, M, N, 2.5, -0.01)
    taken, got = run_stream(x, M, N, grid=grid)
    assert taken == sk.SK_PATH_STREAM
    check(got, want, f"N={N} M={M} F={F} grid={grid}")


def test_stream_path_synthetic_rfi():
    """The synthetic noise and RFI model at a small array (N = 100, M = 100): masks and
    SK bit-exact, and the injected tones flagged."""
    import synth

    ds = synth.Dataset(n_frames=256, M=100, N=100, seed=31,
                       rfi=synth.rfi_plan(31, 256, cw_frac=0.05, pulse_frac=0.05))
    x = ds.generate_cpu()
    want = oracle.flag(x, 100, 100, 3.0, 0.0)
    taken, got = run_stream(x, 100, 100, n_sigma=3.0, delta=0.0)
    assert taken == sk.SK_PATH_STREAM
    check(got, want, "synthetic N=100 M=100")
    assert want["mask"].sum() > 0


@pytest.mark.parametrize("N,M,F", [(100, 100, 21), (7, 33, 50), (64, 256, 12)])
def test_stream_path_independent_estimates(N, M, F):
    """sk_compute_inputs on the stream path: per-input SK^_i and flags bit-exact."""
    dev = _dev()
    rng = np.random.default_rng(N + 3 * M + F)
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
        sk.sk_plan_set_config(plan, rows=16 if M % 32 == 0 else 8, path=sk.SK_PATH_STREAM)
        sk.sk_compute_inputs(plan, d_in, F, sk_in, m_in, skv, mask)
        torch.cuda.synchronize()
        assert sk.sk_plan_get_config(plan)["last_path"] == sk.SK_PATH_STREAM
    finally:
        sk.sk_plan_destroy(plan)
    assert np.array_equal(sk_in.cpu().numpy().view(np.uint32), want["sk_in"].view(np.uint32))
    assert np.array_equal(m_in.cpu().numpy(), want["mask_in"])
    assert np.array_equal(mask.cpu().numpy(), whole["mask"])
    assert np.array_equal(skv.cpu().numpy().view(np.uint32), whole["sk"].view(np.uint32))


def test_stream_path_not_taken_where_it_cannot():
    """N / gcd(N, 16) above 512 (N = 2047) has no stream shape: a request for it takes
    the path the library chooses for the shape (here the ragged row-balanced path), with
    the same results."""
    rng = np.random.default_rng(5)
    N, M, F = 2047, 32, 5
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    taken, got = run_stream(x, M, N)
    _, auto = run_stream(x, M, N, path=sk.SK_PATH_AUTO)
    assert taken == sk.SK_PATH_ROW_BALANCED
    check(got, oracle.flag(x, M, N, 2.5, -0.01), "N=2047 fallback")
    check(auto, oracle.flag(x, M, N, 2.5, -0.01), "N=2047 auto")


@pytest.mark.parametrize("N,M,F,path", [
    (100, 100, 40, sk.SK_PATH_STREAM), (8, 256, 130, sk.SK_PATH_STREAM),
    (100, 256, 20, sk.SK_PATH_STREAM), (64, 100, 30, sk.SK_PATH_STREAM),
    (128, 256, 20, sk.SK_PATH_TEAM), (99, 101, 12, sk.SK_PATH_GENERAL),
    (500, 100, 20, sk.SK_PATH_STREAM), (2044, 100, 4, sk.SK_PATH_STREAM),
    (300, 48, 30, sk.SK_PATH_ROW_BALANCED),
])
def test_auto_path_choice(N, M, F, path):
    """A plan that asks for no path takes the stream path where it measured faster (the
    general path's shapes of any N; below N = 256 also the ragged shapes and the team
    shapes below N = 64) and keeps the others; results bit-exact either way."""
    rng = np.random.default_rng(N + M)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    taken, got = run_stream(x, M, N, path=sk.SK_PATH_AUTO)
    assert taken == path
    check(got, oracle.flag(x, M, N, 2.5, -0.01), f"auto N={N} M={M}")


def test_stream_path_graph_capture_and_host_calls():
    """The stream path inside a captured CUDA graph (replayed twice), through the
    host-buffer call (frames staged in chunks) and through the allocation-free host
    call: the oracle's masks and SK every time."""
    dev = _dev()
    N, M, F = 100, 100, 1500
    rng = np.random.default_rng(77)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    want = oracle.flag(x, M, N, 3.0, 0.0)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    plan = sk.sk_plan_create(N, M, 3.0, 0.0)
    try:
        m1 = torch.full((F,), 7, dtype=torch.uint8, device=dev)
        sk1 = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
        sk.sk_flag(plan, d_in, F, sk1, m1)  # first launch outside the capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sk.sk_flag(plan, d_in, F, sk1, m1, torch.cuda.current_stream())
        for _ in range(2):
            m1.fill_(7)
            sk1.fill_(-1.0)
            g.replay()
        torch.cuda.synchronize()
        assert sk.sk_plan_get_config(plan)["last_path"] == sk.SK_PATH_STREAM
        assert np.array_equal(m1.cpu().numpy(), want["mask"])
        assert np.array_equal(sk1.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32))
        for call in (sk.sk_flag_host, sk.sk_flag_host_noalloc):
            h_sk = np.full(F, -1.0, dtype=np.float32)
            h_mask = np.full(F, 7, dtype=np.uint8)
            call(plan, x, F, h_sk, h_mask)
            assert np.array_equal(h_mask, want["mask"]), call.__name__
            assert np.array_equal(h_sk.view(np.uint32), want["sk"].view(np.uint32)), call.__name__
    finally:
        sk.sk_plan_destroy(plan)


# Input-major frames ([frame][input][t]) of any M: the chunk path (two lanes per input,
# the aligned 16-byte chunks that cover it, neighbours' bytes masked).  (N, M, F, path
# requested): no fast path for these M (auto), and fast-path shapes asked for it.
IMAJOR = [
    (100, 100, 37, 0), (2048, 100, 9, 0), (256, 48, 21, 0), (2048, 200, 5, 0),
    (7, 3, 999, 0), (33, 17, 120, 0), (1, 2, 500, 0), (4096, 5, 40, 0), (100, 1000, 7, 0),
    (3, 4095, 11, 0), (250, 33, 40, 0), (2047, 101, 3, 0), (31, 4096, 2, sk.SK_PATH_STREAM),
    (64, 96, 30, sk.SK_PATH_STREAM), (2048, 256, 4, sk.SK_PATH_STREAM),
    # staged blocks (M <= 192): 4, 8 and 13 chunks a lane, words and 16-byte pieces,
    # a partial last block, one-warp and several-warp teams
    (300, 127, 5, 0), (40, 80, 9, 0), (2048, 36, 3, 0), (65, 192, 4, sk.SK_PATH_STREAM),
    (3, 191, 30, 0), (9, 112, 11, 0), (1000, 63, 6, 0),
]


@pytest.mark.parametrize("N,M,F,path", IMAJOR)
def test_input_major_chunk_path_bit_exact(N, M, F, path):
    """S1, S2, Q, N_eff, SK and masks of the input-major chunk path against the oracle
    (random bytes with nibble 0, a dead frame and a dead input)."""
    dev = _dev()
    rng = np.random.default_rng(N * 131 + M * 7 + F)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    if F > 3:
        x[1] = 0x88
        x[2, :M] = 0x88           # input 0 without power
    want = oracle.flag(x, M, N, 2.5, -0.01, layout=1)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    s1 = torch.full((F, N), -1, dtype=torch.int32, device=dev)
    s2 = torch.full_like(s1, -1)
    q = torch.full((F,), -1, dtype=torch.int64, device=dev)
    skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
    ne = torch.full((F,), -1, dtype=torch.int32, device=dev)
    sk2 = torch.full_like(skv, -1.0)
    mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N, M, 2.5, -0.01, layout=1)
    try:
        if path:
            sk.sk_plan_set_config(plan, path=path)
        sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
        sk.sk_flag(plan, d_in, F, sk2, mask)
        torch.cuda.synchronize()
        assert sk.sk_plan_get_config(plan)["last_path"] == sk.SK_PATH_STREAM
    finally:
        sk.sk_plan_destroy(plan)
    got = dict(S1=s1.cpu().numpy(), S2=s2.cpu().numpy(), Q=q.cpu().numpy(),
               neff=ne.cpu().numpy(), sk=skv.cpu().numpy(), sk_flag=sk2.cpu().numpy(),
               mask=mask.cpu().numpy())
    check(got, want, f"input-major N={N} M={M} F={F}")


@pytest.mark.parametrize("N,M,F", [(100, 100, 21), (2048, 48, 3)])
def test_input_major_chunk_path_independent_estimates(N, M, F):
    """sk_compute_inputs on the input-major chunk path: per-input SK^_i and flags."""
    dev = _dev()
    rng = np.random.default_rng(N + 5 * M + F)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    want = oracle.flag_inputs(x, M, N, 3.0, 0.05, layout=1)
    whole = oracle.flag(x, M, N, 3.0, 0.05, layout=1)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    sk_in = torch.empty((F, N), dtype=torch.float32, device=dev)
    m_in = torch.empty((F, N), dtype=torch.uint8, device=dev)
    mask = torch.empty(F, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N, M, 3.0, 0.05, layout=1)
    try:
        sk.sk_compute_inputs(plan, d_in, F, sk_in, m_in, None, mask)
        torch.cuda.synchronize()
        assert sk.sk_plan_get_config(plan)["last_path"] == sk.SK_PATH_STREAM
    finally:
        sk.sk_plan_destroy(plan)
    assert np.array_equal(sk_in.cpu().numpy().view(np.uint32), want["sk_in"].view(np.uint32))
    assert np.array_equal(m_in.cpu().numpy(), want["mask_in"])
    assert np.array_equal(mask.cpu().numpy(), whole["mask"])


def test_random_stream_and_chunk_shapes():
    """40 seeded random shapes on the stream path (time-major, N up to 600, any M,
    frames at every 16-byte offset) and the input-major chunk path (any M not a multiple
    of 32), random grid sizes, the path asked for or chosen by the library: S1, S2, Q,
    N_eff, SK bits and masks bit-exact against the oracle."""
    dev = _dev()
    rng = np.random.default_rng(1808_10365)
    for case in range(40):
        layout = int(rng.integers(0, 2))
        if layout == 0:
            N = int(rng.integers(1, 601))
            M = int(rng.integers(2, 400))
        else:
            N = int(rng.integers(1, 2500))
            M = int(rng.integers(2, 1200))
            if M % 32 == 0:
                M += 1
        F = int(rng.integers(1, 40))
        while F > 1 and F * M * N > (8 << 20):
            F //= 2
        grid = int(rng.choice([0, 1, 3, 17]))
        path = int(rng.choice([sk.SK_PATH_AUTO, sk.SK_PATH_STREAM]))
        x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
        want = oracle.flag(x, M, N, 2.5, 0.02, layout=layout)
        d_in = torch.from_numpy(x.reshape(-1)).to(dev)
        s1 = torch.full((F, N), -1, dtype=torch.int32, device=dev)
        s2 = torch.full_like(s1, -1)
        q = torch.full((F,), -1, dtype=torch.int64, device=dev)
        skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
        ne = torch.full((F,), -1, dtype=torch.int32, device=dev)
        mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
        plan = sk.sk_plan_create(N, M, 2.5, 0.02, layout=layout)
        try:
            sk.sk_plan_set_config(plan, rows=16 if M % 32 == 0 else 8, grid_ctas=grid, path=path)
            sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
            sk.sk_flag(plan, d_in, F, None, mask)
            torch.cuda.synchronize()
            taken = sk.sk_plan_get_config(plan)["last_path"]
        finally:
            sk.sk_plan_destroy(plan)
        label = f"case {case}: N={N} M={M} F={F} layout={layout} grid={grid} path={path} -> {taken}"
        for k, g in (("S1", s1), ("S2", s2), ("Q", q), ("neff", ne), ("mask", mask)):
            assert np.array_equal(g.cpu().numpy(), want[k]), f"{label}: {k}"
        assert np.array_equal(skv.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32)), label


def test_random_staged_input_major_shapes():
    """30 seeded random input-major shapes of M <= 192 without a fast path (the staged
    blocks: words with and without shifts, 16-byte pieces, whole-block loads with and
    without end checks, the L2 look-ahead from M = 112, partial last blocks), random grid
    sizes and frame counts: S1, S2, Q, N_eff, SK bits and masks bit-exact against the
    oracle, and the path reported as the stream path."""
    dev = _dev()
    rng = np.random.default_rng(2019)
    for case in range(30):
        N = int(rng.choice([int(rng.integers(1, 130)), int(rng.integers(130, 2500))]))
        M = int(rng.integers(2, 193))
        if M % 32 == 0:
            M -= 1
        F = int(rng.integers(1, 60))
        while F > 1 and F * M * N > (8 << 20):
            F //= 2
        grid = int(rng.choice([0, 1, 3, 17]))
        x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
        want = oracle.flag(x, M, N, 2.5, 0.02, layout=1)
        d_in = torch.from_numpy(x.reshape(-1)).to(dev)
        s1 = torch.full((F, N), -1, dtype=torch.int32, device=dev)
        s2 = torch.full_like(s1, -1)
        q = torch.full((F,), -1, dtype=torch.int64, device=dev)
        skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
        ne = torch.full((F,), -1, dtype=torch.int32, device=dev)
        mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
        plan = sk.sk_plan_create(N, M, 2.5, 0.02, layout=1)
        try:
            sk.sk_plan_set_config(plan, rows=8, grid_ctas=grid)
            sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
            sk.sk_flag(plan, d_in, F, None, mask)
            torch.cuda.synchronize()
            taken = sk.sk_plan_get_config(plan)["last_path"]
        finally:
            sk.sk_plan_destroy(plan)
        label = f"case {case}: N={N} M={M} F={F} grid={grid} -> {taken}"
        assert taken == sk.SK_PATH_STREAM, label
        for k, g in (("S1", s1), ("S2", s2), ("Q", q), ("neff", ne), ("mask", mask)):
            assert np.array_equal(g.cpu().numpy(), want[k]), f"{label}: {k}"
        assert np.array_equal(skv.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32)), label

def test_batch_with_stream_and_chunk_classes():
    """A batched launch mixing items of the stream path (small and odd time-major
    shapes), input-major staged blocks (M <= 192) and chunks (8 lanes per input, longer
    M) and a fused-kernel class: one persistent launch per class in one graph, replayed
    twice, every item's SK and mask bit-exact against the oracle."""
    dev = _dev()
    rng = np.random.default_rng(4242)
    shapes = [  # (N, M, layout, F)
        (100, 100, 0, 150), (8, 256, 0, 400), (500, 100, 0, 30), (99, 101, 0, 20),
        (2048, 100, 1, 6), (256, 48, 1, 40), (33, 17, 1, 300), (2048, 256, 0, 12),
        (16, 64, 0, 999), (7, 3, 1, 500), (100, 300, 1, 5), (64, 1000, 1, 3),
    ]
    plans, ins, outs, wants, items = [], [], [], [], []
    try:
        for N, M, layout, F in shapes:
            x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
            wants.append(oracle.flag(x, M, N, 3.0, 0.01, layout=layout))
            plan = sk.sk_plan_create(N, M, 3.0, 0.01, layout=layout)
            plans.append(plan)
            d_in = torch.from_numpy(x.reshape(-1)).to(dev)
            d_sk = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
            d_mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
            ins.append(d_in)
            outs.append((d_sk, d_mask))
            items.append((plan, d_in, F, d_sk, d_mask))
        batch = sk.sk_batch_create(items)
        try:
            # classes: stream (time-major small/odd), staged input-major blocks (M =
            # 100, 48, 17, 3), chunk G = 8 (M = 300, 1000), the general class (N = 99,
            # M = 101 keeps the general path), and N = 2048 (its own fused-kernel class)
            assert sk.sk_batch_launches(batch) >= 5
            for _ in range(2):
                for d_sk, d_mask in outs:
                    d_sk.fill_(-1.0)
                    d_mask.fill_(7)
                sk.sk_batch_run(batch)
                torch.cuda.synchronize()
                for (N, M, layout, F), (d_sk, d_mask), want in zip(shapes, outs, wants):
                    label = f"batch item N={N} M={M} layout={layout}"
                    assert np.array_equal(d_mask.cpu().numpy(), want["mask"]), label
                    assert np.array_equal(d_sk.cpu().numpy().view(np.uint32),
                                          want["sk"].view(np.uint32)), label
        finally:
            sk.sk_batch_destroy(batch)
    finally:
        for p in plans:
            sk.sk_plan_destroy(p)
