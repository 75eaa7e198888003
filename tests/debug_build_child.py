"""Child process of tests/test_debug_build_gpu.py: runs the library's debug build
(SK_DEBUG_LIBRARY=1, loaded by the binding) over small cases of every read path
and checks the results against the oracle; every call would report a failed bounds
check of an earlier launch of its plan.  argv[1] == "shrink": every plan takes its
input as SK_DEBUG_SHRINK_INPUT bytes shorter than it is, so the last loads fail
their checks, and the plan's next call must report it."""

import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402

assert sk.LIB_PATH.endswith("libsk_debug.so"), sk.LIB_PATH
dev = torch.device("cuda:0")


def flag(plan, x, N, M, F, sk_out=True):
    d_in = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(dev)
    skv = torch.full((F,), -1.0, dtype=torch.float32, device=dev)
    mask = torch.full((F,), 7, dtype=torch.uint8, device=dev)
    sk.sk_flag(plan, d_in, F, skv, mask)
    torch.cuda.synchronize()
    return skv.cpu().numpy(), mask.cpu().numpy()


def check_case(N, M, layout, F, cfg=None, seed=0):
    rng = np.random.default_rng(seed + N + M)
    x = rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)
    want = oracle.flag(x, M, N, 3.0, 0.0, layout=layout)
    plan = sk.sk_plan_create(N, M, 3.0, 0.0, layout=layout)
    try:
        if cfg:
            sk.sk_plan_set_config(plan, **cfg)
        got = flag(plan, x, N, M, F)
        taken = sk.sk_plan_get_config(plan)["last_path"]
        assert np.array_equal(got[1], want["mask"]), (N, M, layout, cfg)
        assert np.array_equal(got[0].view(np.uint32), want["sk"].view(np.uint32))
        # sums, Q and N_eff through sk_compute on the same plan
        d_in = torch.from_numpy(x.reshape(-1)).to(dev)
        s1 = torch.empty((F, N), dtype=torch.int32, device=dev)
        s2 = torch.empty_like(s1)
        q = torch.empty(F, dtype=torch.int64, device=dev)
        ne = torch.empty(F, dtype=torch.int32, device=dev)
        sk.sk_compute(plan, d_in, F, s1, s2, q, None, ne)
        torch.cuda.synchronize()
        assert np.array_equal(s1.cpu().numpy(), want["S1"]) and np.array_equal(q.cpu().numpy(), want["Q"])
        # a further call reports any failed check of the launches above
        flag(plan, x[:1], N, M, 1)
        return taken
    finally:
        sk.sk_plan_destroy(plan)


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "shrink":
        N, M, F = 2048, 256, 12
        x = np.full((F, M * N), 0x99, dtype=np.uint8)
        plan = sk.sk_plan_create(N, M, 3.0, 0.0)
        try:
            flag(plan, x, N, M, F)             # its last loads fail their checks
            try:
                flag(plan, x, N, M, F)
            except sk.SkError as e:
                assert e.status == sk.SK_ERR_CUDA and "bounds check" in e.message, e
                print("bounds check reported:", e.message)
                return 0
            raise AssertionError("no bounds report")
        finally:
            sk.sk_plan_destroy(plan)
    T, WS, RB, GEN, PI, ST = (sk.SK_PATH_TEAM, sk.SK_PATH_WARP_SLICE, sk.SK_PATH_ROW_BALANCED,
                              sk.SK_PATH_GENERAL, sk.SK_PATH_PER_INPUT, sk.SK_PATH_STREAM)
    cases = [  # (N, M, layout, F, config or None, path the launch must take)
        (2048, 256, 0, 40, None, RB),
        (2048, 256, 0, 9, dict(path=WS), WS),
        (2048, 256, 0, 9, dict(path=T), T),
        (2048, 48, 0, 21, None, RB),
        (2048, 48, 0, 21, dict(rows=8, path=T), T),
        (256, 256, 0, 700, None, T),
        (1000, 64, 0, 33, None, RB),
        (2056, 64, 0, 33, None, RB),             # folded tail: 8 warps + 8 columns
        (2056, 64, 0, 7, dict(path=WS), WS),
        (264, 96, 0, 31, None, RB),              # one warp + 1 group of 8 columns
        (264, 96, 0, 5, dict(path=WS), WS),
        (2047, 256, 0, 5, None, RB),
        (2047, 256, 0, 5, dict(path=T), GEN),
        (333, 96, 0, 31, None, RB),
        (100, 100, 0, 37, None, ST),             # stream path: one unit a warp
        (100, 100, 0, 37, dict(path=T), GEN),
        (8, 256, 0, 300, None, ST),              # four units a warp
        (250, 200, 0, 9, None, ST),              # units of four warps
        (99, 101, 0, 23, None, GEN),
        (99, 101, 0, 23, dict(path=ST), ST),     # frames at every 16-byte offset
        (2048, 256, 1, 40, None, RB),
        (2048, 256, 1, 9, dict(path=T), T),
        (256, 64, 1, 30, None, T),
        (2048, 64, 1, 30, None, RB),
        (256, 96, 1, 30, None, PI),
        (512, 2048, 1, 6, None, WS),
        (33, 384, 1, 7, None, PI),
        (33, 100, 1, 7, None, ST),               # input-major staged blocks (words)
        (2048, 100, 1, 3, None, ST),             # teams of 16 warps a frame
        (256, 96, 1, 9, dict(path=ST), ST),      # staged 16-byte pieces
        (40, 80, 1, 9, None, ST),
        (100, 300, 1, 5, None, ST),              # input-major chunk path (M > 192)
    ]
    for N, M, layout, F, cfg, path in cases:
        taken = check_case(N, M, layout, F, cfg)
        assert taken == path, (N, M, layout, cfg, taken, path)
    # a batched launch over three fused-kernel classes, the stream class, the staged
    # input-major class and an input-major chunk class
    rng = np.random.default_rng(5)
    shapes = [(2048, 128, 11), (2048, 256, 9), (256, 1024, 13), (2048, 256, 7),
              (100, 100, 40), (99, 101, 9), (2048, 100, 3), (33, 17, 50), (100, 300, 4)]
    layouts = [0, 0, 0, 1, 0, 0, 1, 1, 1]
    xs = [rng.integers(0, 256, size=(F, M * N), dtype=np.uint8) for N, M, F in shapes]
    plans = [sk.sk_plan_create(N, M, 3.0, 0.0, layout=l) for (N, M, F), l in zip(shapes, layouts)]
    d = [torch.from_numpy(x.reshape(-1)).to(dev) for x in xs]
    outs = [(torch.empty(F, dtype=torch.float32, device=dev), torch.empty(F, dtype=torch.uint8, device=dev))
            for N, M, F in shapes]
    b = sk.sk_batch_create([(p, di, F, s, m) for p, di, (N, M, F), (s, m) in zip(plans, d, shapes, outs)], 0)
    sk.sk_batch_run(b)
    torch.cuda.synchronize()
    sk.sk_batch_run(b)  # reports a failed check of the first run
    torch.cuda.synchronize()
    for x, (N, M, F), l, (s, m) in zip(xs, shapes, layouts, outs):
        w = oracle.flag(x, M, N, 3.0, 0.0, layout=l)
        assert np.array_equal(m.cpu().numpy(), w["mask"])
    sk.sk_batch_destroy(b)
    for p in plans:
        sk.sk_plan_destroy(p)
    print("debug build: every case exact, no bounds check failed")
    return 0


if __name__ == "__main__":
    sys.exit(main())
