"""The input generator (published Philox vectors, level distribution, regenerability)
and invariants of the oracle's served-state path."""

import numpy as np

import oracle
import synth
from oracle import digitisation as dg
from oracle import served


def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with the generator (Salmon et al. 2011)."""
    assert list(synth.philox_block([0, 0, 0, 0], [0, 0])) == [
        0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert list(synth.philox_block([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2)) == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert list(synth.philox_block([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                                   [0xA4093822, 0x299F31D0])) == [
        0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_level_distribution_matches_model():
    N, M = 4, 256
    ds = synth.Dataset(n_frames=200, M=M, N=N, seed=42, sigma=np.array([1.52, 2.5, 3.0, 3.5]))
    x = ds.generate_cpu().reshape(200, M, N)
    re = (x >> 4).astype(int) - 8
    for i, s in enumerate(ds.sigma):
        _, p = dg.level_probs(s)
        counts = np.bincount(re[:, :, i].ravel() + 7, minlength=15)
        n = counts.sum()
        # chi-square over the populated levels
        e = np.asarray(p).reshape(-1) * n
        m = e > 20
        chi2 = (((counts[m] - e[m]) ** 2) / e[m]).sum()
        assert chi2 < 60, (s, chi2)


def test_frames_regenerate_alone_and_layouts_transpose():
    ds = synth.pathfinder_config()
    full = ds.generate_cpu()
    part = ds.generate_cpu(frame0=37, n=5)
    assert (full[37:42] == part).all()
    dt = synth.Dataset(n_frames=3, M=16, N=10, seed=5, layout=0)
    di = synth.Dataset(n_frames=3, M=16, N=10, seed=5, layout=1, sigma=dt.sigma)
    a = dt.generate_cpu().reshape(3, 16, 10)
    b = di.generate_cpu().reshape(3, 10, 16)
    assert (a.transpose(0, 2, 1) == b).all()


def test_rfi_plan_disjoint_and_sized():
    r = synth.rfi_plan(synth.sub_seed(1, 0), 1525)
    frames = [x.frame for x in r]
    assert len(frames) == len(set(frames)) == 30 + 15
    assert sum(1 for x in r if x.kind == "cw") == 30
    assert all(1.0 <= x.amp <= 5.0 for x in r)


def test_cw_lowers_and_pulse_raises_sk():
    """CW tones drive SK below 1, a short-duty pulse above 1 (spec RFI checks)."""
    ds = synth.pathfinder_config(duty=0.25)
    r = oracle.flag(ds.generate_cpu(), 256, 256, 3.0, float(np.mean(dg.delta_of_sigma(ds.sigma))))
    clean = np.r_[0:10, 20:40, 45:64]
    base = np.median(r["sk64"][clean])
    assert (r["sk64"][10:20] < base - 0.1).all()
    assert (r["sk64"][40:45] > base + 0.05).all()
    assert (r["mask"][10:20] == 1).all() and (r["mask"][40:45] == 1).all()
    assert r["mask"][clean].sum() <= 2


def _served_setup(T=40, N=32, M=256):
    ds = synth.Dataset(n_frames=T, M=M, N=N, seed=77,
                       rfi=[synth.RFI(5, "cw", 4.0), synth.RFI(6, "cw", 4.0)])
    return ds, ds.generate_cpu(), dg.offset_table(M, B=4096)


def test_served_state_flagged_frames_leave_state():
    ds, x, e = _served_setup()
    M, N = ds.M, ds.N
    full = served.served_flags(x, M, N, e)
    assert full["mask"][5] == 1 and full["mask"][6] == 1
    # dropping the flagged frames changes nothing for the others' state evolution
    keep = [f for f in range(ds.n_frames) if f not in (5, 6)]
    sub = served.served_flags(x[keep], M, N, e)
    assert (sub["P"] == full["P"]).all()
    assert (sub["E"] == full["E"][keep]).all()


def test_served_state_checkpoint_resume():
    ds, x, e = _served_setup()
    M, N = ds.M, ds.N
    full = served.served_flags(x, M, N, e)
    a = served.served_flags(x[:17], M, N, e)
    b = served.served_flags(x[17:], M, N, e, P0=a["P"])
    assert (np.concatenate([a["mask"], b["mask"]]) == full["mask"]).all()
    assert (b["P"] == full["P"]).all()


def test_served_offset_tracks_per_input_sigma():
    """The running state's shift E approaches sum_i delta(sigma_i) in Q units (App. B)."""
    ds, x, e = _served_setup(T=60)
    M, N = ds.M, ds.N
    full = served.served_flags(x, M, N, e)
    want = float(np.sum(dg.delta_of_sigma(ds.sigma))) * 2 ** 32 * (M - 1) / (M + 1)
    got = float(full["E"][-1])
    assert abs(got - want) < 0.05 * abs(want) + 0.002 * 2 ** 32 * N


def test_f32_of_int_rounds_once():
    from oracle.served import f32_of_int

    for v in [0, 1, 2 ** 24 - 1, 2 ** 24 + 1, 2 ** 24 + 3, 2 ** 53 + 2 ** 29 + 1, 3 * 2 ** 60 + 12345,
              2 ** 62 - 1]:
        want = np.float32(np.longdouble(v)) if v < 2 ** 64 else None
        # exact reference: the closer of the two neighbouring fp32 values, ties to even
        got = f32_of_int(v)
        lo = np.nextafter(got, np.float32(0))
        hi = np.nextafter(got, np.float32(np.inf))
        from fractions import Fraction
        d = abs(Fraction(int(got)) - v) if got == int(got) else None
        assert d is not None
        assert d <= abs(Fraction(int(lo)) - v) and d <= abs(Fraction(int(hi)) - v)
        del want


def test_running_mu_first_frame_equals_frame_normalisation():
    """With the state initialised from the frame (mu_i = S1_i/n), Eq. avgSK's general form
    rescaled by Eq. final equals the per-frame estimator."""
    ds = synth.Dataset(n_frames=3, M=256, N=64, seed=3)
    x = ds.generate_cpu()
    e = dg.offset_table(256)
    a = served.served_flags(x[:1], 256, 64, e)
    b = served.served_flags(x[:1], 256, 64, e, running_mu=True)
    assert abs(float(a["sk"][0]) - float(b["sk"][0])) <= 1e-6 * abs(float(a["sk"][0]))


def test_running_mu_sees_a_power_step():
    """Half the inputs jump in power against their running state: the running-mu
    estimator moves by about 2 N sum(l^2)/(sum l)^2 - 1 (l the power ratios), the
    per-frame normalisation does not."""
    M, N, T = 256, 128, 30
    sig = np.full(N, 1.6)
    ds1 = synth.Dataset(n_frames=T, M=M, N=N, seed=41, sigma=sig)
    sig2 = sig.copy()
    sig2[: N // 2] *= np.sqrt(2.0)          # power x2 on half of the inputs
    ds2 = synth.Dataset(n_frames=T, M=M, N=N, seed=42, sigma=sig2)
    x = np.concatenate([ds1.generate_cpu(), ds2.generate_cpu()[:1]])
    e = dg.offset_table(M)
    rm = served.served_flags(x, M, N, e, running_mu=True)
    pf = served.served_flags(x, M, N, e)
    lam = np.where(np.arange(N) < N // 2, 2.0, 1.0)
    want = 2 * N * (lam ** 2).sum() / lam.sum() ** 2 - 1      # 1 + 1/9 for this split
    step_rm = float(rm["sk"][-1]) - float(np.mean(rm["sk"][T - 10:T]))
    step_pf = float(pf["sk"][-1]) - float(np.mean(pf["sk"][T - 10:T]))
    # quantisation makes the power ratio and the kurtosis of the stepped inputs differ a
    # little from the continuous-Gaussian closed form: a coarse band around it
    assert 0.6 * (want - 1.0) < step_rm < 1.2 * (want - 1.0)
    assert abs(step_pf) < 0.04
    assert rm["mask"][-1] == 1 and pf["mask"][-1] == 0


def test_repeated_frame_is_a_fixed_point_of_the_state():
    """One frame served again and again: P = 2^6 S1 is the leaky integrator's fixed
    point (P - P/64 + S1 = P exactly in integers), so the state never moves and every
    frame gets the first frame's SK, E and mask, in both normalisations."""
    M, N, T = 256, 64, 8
    x1 = synth.Dataset(n_frames=1, M=M, N=N, seed=5).generate_cpu()
    x = np.repeat(x1, T, axis=0)
    e = dg.offset_table(M)
    for rm in (False, True):
        r = served.served_flags(x, M, N, e, running_mu=rm)
        S1 = r["S1"][0] if np.ndim(r["S1"]) == 2 else r["S1"]
        assert np.array_equal(np.asarray(r["P"], dtype=np.int64),
                              np.asarray(S1, dtype=np.int64) << 6)
        assert np.all(r["sk"].view(np.uint32) == r["sk"][0].view(np.uint32))
        assert np.all(r["mask"] == r["mask"][0]) and np.all(r["E"] == r["E"][0])


def test_running_mu_against_exact_rationals():
    """The running-mu estimator of the served oracle (its 2^24 fixed-point sums and
    double-precision steps) against the exact rational statement of Eq. (avgSK) 1st
    line with mu_i = P_i / (2^6 n), rescaled by Eq. (final) 1st line (brute.py), on
    tiny arrays with random bytes (nibble 0 included) and random states.

    Error bound: a_i and b_i carry at most three fp32 roundings each (two
    conversions and the divide, 2^-24 relative apiece), so X = n' B / A^2 is within
    about 6e-7 relative of its exact value, and SK~ = (n+1)/(n-1) (X - 1) within
    (n+1)/(n-1) 6e-7 X; the fixed-point rounding (2^-25 per term) is far below."""
    from fractions import Fraction

    from oracle import brute

    rng = np.random.default_rng(1808)
    k = 6
    worst = 0.0
    for case in range(120):
        M = int(rng.integers(2, 17))
        N = int(rng.integers(1, 9))
        x = rng.integers(0, 256, size=M * N, dtype=np.uint8)
        if case % 7 == 0:
            x[0::N] = 0x88                      # input 0 has no power
        S1, S2 = brute.sums(x, M, N)
        P = []
        for s1 in S1:
            base = s1 if s1 > 0 else int(rng.integers(1, 60))
            P.append(max(1, int(round(base * (1 << k) * 2.0 ** rng.uniform(-2.0, 2.0)))))
        A, B, ne, skd = served._running_mu_sk(np.array(S1, dtype=np.int64),
                                             np.array(S2, dtype=np.int64),
                                             np.array(P, dtype=np.int64), M, k)
        mu = [Fraction(p, (1 << k) * M) for p in P]
        want, ne_w, ratio = brute.sk_running_mu(S1, S2, mu, M)
        assert ne == ne_w
        if want is None:
            assert skd != skd
            continue
        err = abs(skd - float(want))
        tol = (M + 1) / (M - 1) * 1e-6 * float(ratio) + 1e-9
        worst = max(worst, err / tol)
        assert err <= tol, (case, M, N, skd, float(want))
    assert worst < 1.0


def test_bucket_edges_from_mean_power():
    """bucket(P) is the index b of the power bucket [b, b+1) * 128 / B that holds the
    running mean power per sample mu = P / (2^k n): checked at both sides of every
    bucket edge found by exact rationals, at n where P * B exceeds 2^32 (n = 4096),
    at the top (mu >= 128 clips to B - 1) and at P = 0."""
    from fractions import Fraction

    B, k = 4096, 6
    rng = np.random.default_rng(3)
    wide = 0
    for M in (2, 16, 256, 1024, 4096):
        scale = (1 << k) * M
        edges = sorted(set([1, 2, B - 1] + rng.integers(1, B, 40).tolist()))
        for b in edges:
            # smallest P with P / scale >= b * 128 / B
            lo = Fraction(b * 128, B) * scale
            p_edge = lo.numerator // lo.denominator + (lo.denominator != 1)
            got = served.bucket(np.array([p_edge - 1, p_edge], dtype=np.int64), M, B, k)
            assert got.tolist() == [b - 1, b], (M, b)
            wide += p_edge * B > 2 ** 32              # the uint64 product path
        top = served.bucket(np.array([128 * scale - 1, 128 * scale, 2 ** 32 - 1, 0],
                                     dtype=np.int64), M, B, k)
        assert top.tolist() == [B - 1, B - 1, B - 1, 0]
    assert wide >= 20


def test_offset_table_against_quadrature():
    """The offset table e[b] (the App. B digitisation offset of bucket b's mean power,
    in Q units) against an independent computation at a spread of buckets: the
    moments of clip(round(sigma g), -7, 7) by adaptive quadrature of the normal
    density over each level's interval (scipy.integrate.quad, not the erfc tail
    formula), sigma solved by Brent's method (not bisection), and the Q-unit scale
    taken from the threshold recipe itself: e[b] must equal the shift of the one-input
    upper threshold when the centre moves by delta (Sec. 3.2 interval in Q units)."""
    import math

    from scipy import integrate, optimize

    def moments_quad(sigma):
        pdf = lambda t: math.exp(-0.5 * (t / sigma) ** 2) / (sigma * math.sqrt(2 * math.pi))
        m2 = m4 = 0.0
        for v in range(1, 8):
            a = v - 0.5
            b = v + 0.5 if v < 7 else math.inf
            p = integrate.quad(pdf, a, b, epsabs=1e-15, epsrel=1e-13, limit=200)[0]
            m2 += 2 * p * v ** 2
            m4 += 2 * p * v ** 4
        return m2, m4

    M = 256
    e = dg.offset_table(M)
    # buckets above 2 m2(inf) = 98 (all samples clipped to +-7) have no sigma: the
    # table clamps them to sigma = 1000 (delta near -1, two-level data)
    for b in (3, 40, 300, 700, 1500, 2200, 3000, 3100, 3600, 4095):
        mu = (b + 0.5) * 128 / 4096
        if mu < 98.0:
            sig = optimize.brentq(lambda s: 2 * moments_quad(s)[0] - mu, 1e-2, 1e3,
                                  xtol=1e-14, rtol=1e-15, maxiter=500)
        else:
            sig = 1000.0
        m2, m4 = moments_quad(sig)
        delta = m4 / (2 * m2 * m2) - 1.5
        lo0, hi0 = oracle.thresholds(M, 1, 3.0, 0.0)
        lo1, hi1 = oracle.thresholds(M, 1, 3.0, delta)
        assert abs(int(e[b]) - int(hi1[1] - hi0[1])) <= 2, (b, int(e[b]), int(hi1[1] - hi0[1]))
        assert abs(int(e[b]) - int(lo1[1] - lo0[1])) <= 2


def test_offset_table_monte_carlo():
    """Two buckets of the table against a Monte Carlo run: complex samples with
    components round(sigma g) clipped to [-7, 7], sigma chosen so the mean power per
    sample is the bucket's centre; the sample kurtosis E|x|^4 / (E|x|^2)^2 - 2 is the
    large-n offset of SK (App. B), 4e6 samples."""
    rng = np.random.default_rng(11)
    M = 256
    e = dg.offset_table(M)
    scale = 2 ** 32 * (M - 1) / (M + 1)
    for b in (900, 2600):
        mu = (b + 0.5) * 128 / 4096
        sig = float(dg.sigma_of_power(mu)[0])
        v = np.clip(np.round(sig * rng.standard_normal((2, 4_000_000))), -7, 7)
        p = v[0] ** 2 + v[1] ** 2
        assert abs(p.mean() - mu) < 0.01 * mu
        d_mc = (p ** 2).mean() / p.mean() ** 2 - 2.0
        assert abs(float(e[b]) / scale - d_mc) < 0.01 * (1 + abs(d_mc)) * 0.3, (b, d_mc)
