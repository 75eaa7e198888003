"""Row-balanced launches: a one-item time-major launch of the warp-slice shapes
hands every team an equal range of 32-row turns (16-row turns when M = 16 mod
32; an input-major one, of group rows), and frames cut by a range boundary are combined through the plan's
scratch in device memory.  Against the
oracle: cut frames of every kind (a frame shared by two teams, a frame spread
over many teams, a team inside one frame), per-input outputs written by the
warp that completes a column, folded tails (groups of 8 columns past the last
whole slice), one plan on two streams, a captured launch (which hands out whole
frames), and the no-allocation call before and after the plan has its scratch."""

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


def _bytes(N, M, F, seed):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    if F > 1:
        x[1, : N * 4] = 0x88          # a few dead rows
        x[F - 1, :] = 0x00            # a frame of -8-8j everywhere
    return x


@pytest.mark.parametrize("N,M,F,layout", [
    (2048, 256, 299, 0),    # 299 frames over 296 teams: most frames cut in two
    (2048, 1024, 37, 0),    # frames spread over 8 teams each
    (4096, 4096, 3, 0),     # 384 turns over 148 teams: several teams inside a frame
    (512, 4096, 5, 0),      # 640 turns over 640 two-warp teams: one turn each
    (1024, 32, 3001, 0),    # one turn per frame
    (4096, 96, 150, 0),     # 3 turns per frame
    (512, 64, 1, 0),        # fewer turns than teams
    (768, 256, 101, 0),     # 3-warp teams, 5 per CTA (one warp idle)
    (1040, 64, 61, 0),      # a last slice of 16 columns: lanes past N idle
    (1536, 96, 29, 0),      # 6-warp teams, 2 per CTA
    (3008, 32, 17, 0),      # 12-warp teams, one per CTA
    (528, 128, 9, 0),       # 3 warps, the last one with 2 of 32 lanes busy
    (1000, 64, 61, 0),      # N = 8 mod 16: no tensor map, no L2 prefetch
    (2056, 32, 33, 0),
    (3000, 96, 11, 0),
    (256, 256, 64, 0),      # one-warp teams, 16 per CTA: 512 turns over 2368 teams
    (256, 128, 3001, 0),
    (264, 64, 77, 0),       # two warps, the second with one lane busy
    # M = 16 mod 32: 16-row turns on the 8-row tile (the prefetch box every other turn)
    (2048, 48, 301, 0),     # 3 turns per frame, frames cut in every position
    (512, 16, 2999, 0),     # one turn per frame
    (4096, 112, 5, 0),      # 35 turns over 148 teams: fewer turns than teams
    (1000, 80, 61, 0),      # N = 8 mod 16: no tensor map, no prefetch
    (2056, 48, 31, 0),
    # ragged N (not a multiple of 8): unaligned rows, two aligned words and a shift per
    # row, one loop per N mod 8; the last lane holds columns past N
    (2047, 256, 23, 0),     # N mod 8 = 7
    (2049, 64, 99, 0),      # N mod 8 = 1, a last slice of one column
    (1001, 48, 61, 0),      # 5
    (333, 128, 77, 0),      # 5, one team of two warps
    (98, 96, 301, 0),       # 2, one warp with 13 lanes busy
    (4094, 16, 57, 0),      # 6, one turn per frame
    (4093, 112, 3, 0),      # 5, fewer turns than teams
    (3, 32, 700, 0),        # one lane, 3 inputs
    (12, 256, 40, 0),       # 4: every other row on a 4-byte boundary
    (2051, 32, 9, 0),       # 3
    # input-major: group rows of team*M bytes balanced over the grid (M = 128,
    # 256 and 4096; other M hand out whole frames)
    (2048, 256, 299, 1),    # 8 group rows per frame
    (2048, 4096, 3, 1),     # sub-inputs: 8 per input
    (2048, 64, 301, 1),     # groups of 4 inputs on 4 lanes, 64-thread teams
    (256, 64, 999, 1),
    (4096, 128, 150, 1),
    (512, 1024, 37, 1),
    (256, 512, 7, 1)])
def test_cut_frames_bit_exact(N, M, F, layout):
    dev = _dev()
    x = _bytes(N, M, F, N + 7 * M + F)
    want = oracle.flag(x, M, N, 3.0, 0.02, layout=layout)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    s1 = torch.full((F, N), -1, dtype=torch.int32, device=dev)
    s2 = torch.full_like(s1, -1)
    q = torch.full((F,), -1, dtype=torch.int64, device=dev)
    skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
    ne = torch.full((F,), -1, dtype=torch.int32, device=dev)
    mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N, M, 3.0, 0.02, layout=layout)
    try:
        for _ in range(3):   # the scratch is left zero for the next launch
            sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
            sk.sk_flag(plan, d_in, F, None, mask)
            torch.cuda.synchronize()
            assert np.array_equal(s1.cpu().numpy(), want["S1"])
            assert np.array_equal(s2.cpu().numpy(), want["S2"])
            assert np.array_equal(q.cpu().numpy(), want["Q"])
            assert np.array_equal(ne.cpu().numpy(), want["neff"])
            assert np.array_equal(skv.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32))
            assert np.array_equal(mask.cpu().numpy(), want["mask"])
        # per-input estimates on the same cut frames
        wi = oracle.flag_inputs(x, M, N, 3.0, 0.02, layout=layout)
        sk_in = torch.empty((F, N), dtype=torch.float32, device=dev)
        m_in = torch.empty((F, N), dtype=torch.uint8, device=dev)
        sk.sk_compute_inputs(plan, d_in, F, sk_in, m_in)
        torch.cuda.synchronize()
        assert np.array_equal(sk_in.cpu().numpy().view(np.uint32), wi["sk_in"].view(np.uint32))
        assert np.array_equal(m_in.cpu().numpy(), wi["mask_in"])
    finally:
        sk.sk_plan_destroy(plan)


@pytest.mark.parametrize("N,M,F", [
    (2056, 256, 301),   # 8 warps and one folded group of 8 columns: two teams per CTA
    (520, 256, 97),     # 2 warps + 1 group
    (2064, 256, 41),    # 2 groups, with the tensor map's L2 prefetch (N = 0 mod 16)
    (2080, 64, 61),     # 4 groups over 8 warps
    (264, 96, 123),     # one-warp teams and one group
    (288, 96, 123),     # 4 groups > 1 warp: not folded, a second warp of 32 columns
    (776, 48, 77),      # 3 warps + 1 group, 16-row turns on the 8-row tile
    (3848, 32, 9),      # 15 warps + 1 group: one team per CTA, one turn per frame
    (264, 4096, 3),     # 1 warp + 1 group, frames spread over many teams
])
@pytest.mark.parametrize("path", ["balanced", "whole"])
def test_folded_tail_bit_exact(N, M, F, path):
    """N = 256 W + 8 NT (NT of 1..min(4, W)): teams of W warps read the NT groups
    of 8 columns past the last whole slice row-per-lane, one warp per group and frame
    (rotating with the frame): inside the turn loop with balanced rows (frames cut
    between teams, the groups' sums through the scratch), at the frame's end with
    whole frames per team.  S1, S2, Q, N_eff, SK bits, masks and the per-input
    estimates against the oracle."""
    dev = _dev()
    x = _bytes(N, M, F, N + 3 * M + F)
    want = oracle.flag(x, M, N, 3.0, 0.02)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    s1 = torch.full((F, N), -1, dtype=torch.int32, device=dev)
    s2 = torch.full_like(s1, -1)
    q = torch.full((F,), -1, dtype=torch.int64, device=dev)
    skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
    ne = torch.full((F,), -1, dtype=torch.int32, device=dev)
    mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
    plan = sk.sk_plan_create(N, M, 3.0, 0.02)
    try:
        sk.sk_plan_set_config(plan, rows=16 if M % 32 == 0 else 8,
                              path=sk.SK_PATH_WARP_SLICE if path == "whole"
                              else sk.SK_PATH_ROW_BALANCED)
        for _ in range(2):
            sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
            sk.sk_flag(plan, d_in, F, None, mask)
            torch.cuda.synchronize()
            assert np.array_equal(s1.cpu().numpy(), want["S1"])
            assert np.array_equal(s2.cpu().numpy(), want["S2"])
            assert np.array_equal(q.cpu().numpy(), want["Q"])
            assert np.array_equal(ne.cpu().numpy(), want["neff"])
            assert np.array_equal(skv.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32))
            assert np.array_equal(mask.cpu().numpy(), want["mask"])
        assert sk.sk_plan_get_config(plan)["last_path"] == (
            sk.SK_PATH_ROW_BALANCED if path == "balanced" else sk.SK_PATH_WARP_SLICE)
        wi = oracle.flag_inputs(x, M, N, 3.0, 0.02)
        sk_in = torch.empty((F, N), dtype=torch.float32, device=dev)
        m_in = torch.empty((F, N), dtype=torch.uint8, device=dev)
        sk.sk_compute_inputs(plan, d_in, F, sk_in, m_in)
        torch.cuda.synchronize()
        assert np.array_equal(sk_in.cpu().numpy().view(np.uint32), wi["sk_in"].view(np.uint32))
        assert np.array_equal(m_in.cpu().numpy(), wi["mask_in"])
    finally:
        sk.sk_plan_destroy(plan)


def test_one_plan_on_two_streams():
    """Launches of one plan on two streams take turns on the scratch."""
    dev = _dev()
    N, M = 2048, 128
    xs = [_bytes(N, M, F, 100 + F) for F in (301, 97, 450)]
    wants = [oracle.flag(x, M, N, 2.5, 0.0)["mask"] for x in xs]
    d_ins = [torch.from_numpy(x.reshape(-1)).to(dev) for x in xs]
    streams = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    plan = sk.sk_plan_create(N, M, 2.5, 0.0)
    try:
        masks = [torch.full((x.shape[0],), 7, dtype=torch.uint8, device=dev) for x in xs]
        for rep in range(4):
            for k, (d_in, m) in enumerate(zip(d_ins, masks)):
                sk.sk_flag(plan, d_in, xs[k].shape[0], None, m, streams[(k + rep) % 2])
        torch.cuda.synchronize()
        for m, w in zip(masks, wants):
            assert np.array_equal(m.cpu().numpy(), w)
    finally:
        sk.sk_plan_destroy(plan)


@pytest.mark.parametrize("N,M,F", [(2048, 256, 299), (2047, 64, 77), (2056, 64, 41)])
def test_captured_launch_hands_out_whole_frames(N, M, F):
    """A launch captured into a CUDA graph does not use the scratch (a ragged N then
    takes the general path); the replayed graph and the plain launch give the
    oracle's results."""
    dev = _dev()
    x = _bytes(N, M, F, 5)
    want = oracle.flag(x, M, N, 3.0, 0.0)
    d_in = torch.from_numpy(x.reshape(-1)).to(dev)
    plan = sk.sk_plan_create(N, M, 3.0, 0.0)
    try:
        m0 = torch.full((F,), 7, dtype=torch.uint8, device=dev)
        sk.sk_flag(plan, d_in, F, None, m0)      # plain launch: allocates the scratch
        torch.cuda.synchronize()
        m1 = torch.full((F,), 7, dtype=torch.uint8, device=dev)
        sk1 = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sk.sk_flag(plan, d_in, F, sk1, m1, torch.cuda.current_stream())
        for _ in range(2):
            m1.fill_(7)
            g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(m0.cpu().numpy(), want["mask"])
        assert np.array_equal(m1.cpu().numpy(), want["mask"])
        assert np.array_equal(sk1.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32))
    finally:
        sk.sk_plan_destroy(plan)


def test_no_alloc_call_before_and_after_scratch():
    """The no-allocation call balances rows only once the plan has its scratch
    from an earlier call; either way its results are the oracle's."""
    _dev()
    N, M, F = 2048, 256, 31
    x = _bytes(N, M, F, 11)
    want = oracle.flag(x, M, N, 3.0, 0.0)
    plan = sk.sk_plan_create(N, M, 3.0, 0.0)
    try:
        for _ in range(2):   # first without scratch, then with the scratch of sk_flag_host
            h_sk = np.full(F, -1.0, dtype=np.float32)
            h_mask = np.full(F, 7, dtype=np.uint8)
            sk.sk_flag_host_noalloc(plan, x, F, h_sk, h_mask)
            assert np.array_equal(h_mask, want["mask"])
            assert np.array_equal(h_sk.view(np.uint32), want["sk"].view(np.uint32))
            sk.sk_flag_host(plan, x, F, np.zeros(F, dtype=np.float32), np.zeros(F, dtype=np.uint8))
    finally:
        sk.sk_plan_destroy(plan)


def test_random_balanced_shapes_sweep():
    """40 seeded random shapes on the balanced paths (N a multiple of 8 from 256 to
    4096, M a multiple of 32 or, every fourth case, 16 mod 32, 1 to a few hundred frames, so frames cut between
    teams in every way; some input-major with M = 128 or 256), each against the
    oracle: S1, S2, Q, N_eff, SK bits and masks."""
    dev = _dev()
    rng = np.random.default_rng(18081036)
    for case in range(40):
        layout = 1 if rng.random() < 0.2 else 0
        if layout == 0:
            N = int(8 * rng.integers(32, 513))
            M = int(32 * rng.integers(1, 33)) if case % 4 else int(16 * (2 * rng.integers(0, 16) + 1))
        else:
            N = int(256 * rng.integers(1, 9))
            M = int(rng.choice([128, 256]))
        F = int(rng.integers(1, 400))
        while F > 1 and F * M * N > (24 << 20):
            F //= 2
        x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
        want = oracle.flag(x, M, N, 2.5, 0.01, layout=layout)
        d_in = torch.from_numpy(x.reshape(-1)).to(dev)
        s1 = torch.full((F, N), -1, dtype=torch.int32, device=dev)
        s2 = torch.full_like(s1, -1)
        q = torch.full((F,), -1, dtype=torch.int64, device=dev)
        skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
        ne = torch.full((F,), -1, dtype=torch.int32, device=dev)
        mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
        plan = sk.sk_plan_create(N, M, 2.5, 0.01, layout=layout)
        try:
            sk.sk_compute(plan, d_in, F, s1, s2, q, skv, ne)
            sk.sk_flag(plan, d_in, F, None, mask)
            torch.cuda.synchronize()
        finally:
            sk.sk_plan_destroy(plan)
        tag = f"case {case}: N={N} M={M} F={F} layout={layout}"
        assert np.array_equal(s1.cpu().numpy(), want["S1"]), tag
        assert np.array_equal(s2.cpu().numpy(), want["S2"]), tag
        assert np.array_equal(q.cpu().numpy(), want["Q"]), tag
        assert np.array_equal(ne.cpu().numpy(), want["neff"]), tag
        assert np.array_equal(skv.cpu().numpy().view(np.uint32), want["sk"].view(np.uint32)), tag
        assert np.array_equal(mask.cpu().numpy(), want["mask"]), tag
