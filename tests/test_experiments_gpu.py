"""The paper's synthetic experiments, run through the CUDA path (sk_compute), with
the oracle checking the same bytes.

* App. A: a common-mode signal shared by all receivers raises var(SK~) from
  4/(nN) towards the single-receiver value; N_eff = 4/(n var) falls from N to ~1.
* App. B: 4+4-bit data at CHIME-like rms 1.52 LSB: the mean of SK~ sits a small
  constant below 1 (the digitisation offset) and the variance matches the
  unquantised case.
* Sec. 3.2 / Fig. heatmap: the detection significance of the same interference
  grows as sqrt(N) between a 2048- and a 256-input array.
"""

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1808_10365_b300 as sk  # noqa: E402
import synth  # noqa: E402
from oracle import digitisation as dg  # noqa: E402

pytestmark = pytest.mark.gpu


def _gpu_sk(x, M, N):
    """SK~ (fp32) and Q per frame from the CUDA path."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dev = torch.device("cuda:0")
    F = x.shape[0]
    d_in = torch.from_numpy(np.ascontiguousarray(x).reshape(-1)).to(dev)
    skv = torch.empty(F, dtype=torch.float32, device=dev)
    q = torch.empty(F, dtype=torch.int64, device=dev)
    plan = sk.sk_plan_create(N, M)
    try:
        sk.sk_compute(plan, d_in, F, None, None, q, skv, None)
        torch.cuda.synchronize()
    finally:
        sk.sk_plan_destroy(plan)
    return skv.cpu().numpy().astype(np.float64), q.cpu().numpy()


def _quantise(z):
    re = np.clip(np.rint(z.real), -7, 7).astype(np.int64)
    im = np.clip(np.rint(z.imag), -7, 7).astype(np.int64)
    return (((re + 8) << 4) | (im + 8)).astype(np.uint8)


def test_common_mode_raises_variance_app_a():
    M, N, F = 256, 64, 300
    rng = np.random.default_rng(1808)
    ratios, neffs = [], []
    for c in (0.0, 0.3, 1.0, 3.0, 10.0):
        g = rng.standard_normal((F, M, N)) + 1j * rng.standard_normal((F, M, N))
        h = rng.standard_normal((F, M, 1)) + 1j * rng.standard_normal((F, M, 1))
        x = _quantise((g + c * h) * (2.0 / math.sqrt(1.0 + c * c))).reshape(F, -1)
        skv, q = _gpu_sk(x, M, N)
        w = oracle.flag(x[:20], M, N)
        assert np.array_equal(q[:20], w["Q"])
        v = skv.var()
        ratios.append(v / (4.0 / (M * N)))
        neffs.append(4.0 / (M * v))
    assert 0.7 < ratios[0] < 1.3            # independent receivers: 4/(nN)
    assert all(b > a * 0.9 for a, b in zip(ratios, ratios[1:]))
    assert neffs[-1] < 3.0                  # common mode dominates: about one receiver


def test_digitisation_offset_and_variance_app_b():
    M, N, F, s = 256, 1024, 200, 1.52
    ds = synth.Dataset(n_frames=F, M=M, N=N, seed=11, sigma=np.full(N, s))
    x = ds.generate_cpu()
    skv, q = _gpu_sk(x, M, N)
    w = oracle.flag(x[:10], M, N)
    assert np.array_equal(q[:10], w["Q"])
    se = skv.std() / math.sqrt(F)
    d = float(dg.delta_of_sigma(s))
    assert abs((skv.mean() - 1.0) - d) < 5 * se + 0.5 / M   # slightly below 1
    rng = np.random.default_rng(3)
    vf = np.concatenate([oracle.sk_from_complex(rng.standard_normal((50, M, N)) +
                                                1j * rng.standard_normal((50, M, N)))
                         for _ in range(4)]).var()
    assert 0.75 < skv.var() / vf < 1.35                       # variance unchanged


def test_significance_scales_as_sqrt_n():
    M, A, F = 256, 1.0, 60
    sig = {}
    for N in (2048, 256):
        rfi = [synth.RFI(f, "cw", A) for f in range(30, F)]
        ds = synth.Dataset(n_frames=F, M=M, N=N, seed=21 + N, sigma=np.full(N, 2.5), rfi=rfi)
        x = ds.generate_cpu()
        skv, q = _gpu_sk(x, M, N)
        w = oracle.flag(x[28:32], M, N)
        assert np.array_equal(q[28:32], w["Q"])
        centre = skv[:30].mean()
        sig[N] = np.mean((skv[30:] - centre) / (2.0 / math.sqrt(M * N)))
    ratio = sig[2048] / sig[256]
    assert abs(ratio / math.sqrt(2048 / 256) - 1.0) < 0.12
