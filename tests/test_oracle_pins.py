"""Pins of the oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  The oracle is never compared with
itself by retyping its formula: the references are exact rationals, closed
forms, invariants and moments.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import brute
from oracle import digitisation as dg


def _random_bytes(rng, F, M, N):
    return rng.integers(0, 256, size=(F, M * N), dtype=np.uint8)


# --------------------------------------------------------------------------
# brute force on tiny arrays: Eq. 1, Eqs. normedSum1/2, avgSK, final
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M,N,layout", [(2, 1, 0), (3, 5, 0), (16, 8, 0), (7, 3, 1), (16, 8, 1)])
def test_sums_and_sk_against_exact_rationals(M, N, layout):
    rng = np.random.default_rng(1000 + 17 * M + N + layout)
    x = _random_bytes(rng, 6, M, N)      # every byte value possible, nibble 0 (-8) included
    S1, S2 = oracle.power_sums(x, M, N, layout)
    Q, ne, sk32 = oracle.sk_spec(S1, S2, M)
    sk64, s1bar, ne64 = oracle.sk_f64(S1, S2, M)
    for f in range(x.shape[0]):
        bs1, bs2 = brute.sums(list(x[f]), M, N, layout)
        assert list(S1[f]) == bs1 and list(S2[f]) == bs2
        sk_n, sb1, sb2, bne = brute.sk_normalised(bs1, bs2, M)
        assert bne == ne[f] == ne64[f]
        if bne == 0:
            assert np.isnan(sk32[f]) and np.isnan(sk64[f])
            continue
        # Eq. normedSum1: S1bar = n N exactly
        assert sb1 == M * bne
        # Eq. final, lines 2 and 3 agree exactly; Eq. avgSK rescaled by Eq. final line 1 too
        assert sk_n == brute.sk_average(bs1, bs2, M)
        assert brute.rescale_hat(brute.sk_combined_hat(bs1, bs2, M), M, bne) == sk_n
        # Eq. normedSimplifiedSum2: S2bar = n(n-1)/(n+1) sum SK^_i + nN
        ssum = sum((brute.sk_single(a, b, M) for a, b in zip(bs1, bs2) if a), Fraction(0))
        assert sb2 == Fraction(M * (M - 1), M + 1) * ssum + M * bne
        exact = float(sk_n)
        assert abs(sk64[f] - exact) <= 1e-12 * max(1.0, abs(exact))
        assert abs(s1bar[f] - M * bne) <= 1e-9 * M * bne
        # fp32 SK within 1e-6 relative (plus an absolute floor near SK = 0)
        assert abs(float(sk32[f]) - exact) <= 1e-6 * abs(exact) + 1e-9
        # Q is 2^32 * sum r_i up to one fp32 divide per input and rounding to integers
        rsum = sum((Fraction(M * b, a * a) - 1 for a, b in zip(bs1, bs2) if a), Fraction(0))
        rmax = max((Fraction(M * b, a * a) - 1 for a, b in zip(bs1, bs2) if a))
        tol = bne * (0.5 + float(rmax) * 2.0 ** 32 * 3 * 2.0 ** -24)
        assert abs(int(Q[f]) - float(rsum * 2 ** 32)) <= tol


def test_layouts_are_transposes():
    rng = np.random.default_rng(7)
    M, N = 12, 5
    x = _random_bytes(rng, 3, M, N)
    xt = x.reshape(3, M, N).transpose(0, 2, 1).reshape(3, M * N)
    a = oracle.power_sums(x, M, N, 0)
    b = oracle.power_sums(np.ascontiguousarray(xt), M, N, 1)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()


def test_unpack_levels_and_nibble_minus_eight():
    # byte 0x00 is (-8, -8): |x|^2 = 128; 0x88 is (0, 0); 0xF0 is (7, -8)
    for b, p in [(0x00, 128), (0x88, 0), (0xF0, 49 + 64), (0x9A, 1 + 4), (0x7F, 1 + 49)]:
        x = np.array([[b, b]], dtype=np.uint8)   # M=2, N=1
        S1, S2 = oracle.power_sums(x, 2, 1)
        assert S1[0, 0] == 2 * p and S2[0, 0] == 2 * p * p


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def _pack(re, im):
    return ((np.asarray(re) + 8) << 4 | (np.asarray(im) + 8)).astype(np.uint8)


def test_constant_modulus_gives_zero():
    """|x| constant over the frame: n S2 = S1^2, so SK^_i = 0 (Eq. originalSK)."""
    M, N = 64, 9
    rng = np.random.default_rng(3)
    # (3,4), (-4,3), (5,0), (0,-5)... all |x|^2 = 25, phases vary per sample and input
    choices = np.array([(3, 4), (-4, 3), (5, 0), (0, -5), (-3, -4), (4, -3)])
    idx = rng.integers(0, len(choices), size=(2, M, N))
    x = _pack(choices[idx, 0], choices[idx, 1]).reshape(2, M * N)
    r = oracle.flag(x, M, N)
    assert (r["Q"] == 0).all() and (r["sk"] == 0).all() and (r["sk64"] == 0).all()


@pytest.mark.parametrize("M,k", [(256, 128), (256, 64), (256, 1), (100, 37), (2, 1), (1024, 1000)])
def test_on_off_duty_closed_form(M, k):
    """Power P for k of n samples, 0 otherwise: SK^ = (n+1)/(n-1) (n/k - 1) (Eq. originalSK)."""
    N = 4
    re = np.zeros((M, N), dtype=int)
    im = np.zeros((M, N), dtype=int)
    re[:k, :] = 3
    im[:k, :] = -2
    x = _pack(re, im).reshape(1, M * N)
    r = oracle.flag(x, M, N)
    want = (M + 1) / (M - 1) * (M / k - 1)
    assert abs(r["sk64"][0] - want) <= 1e-12 * max(1, want)
    assert abs(float(r["sk"][0]) - want) <= 1e-6 * max(1e-3, want)


def test_single_receiver_matches_eq_sk():
    """N = 1: SK~ is the single-receiver SK^ of Eq. (eq:sk)."""
    rng = np.random.default_rng(11)
    M = 256
    x = _random_bytes(rng, 20, M, 1)
    S1, S2 = oracle.power_sums(x, M, 1)
    sk64, _, _ = oracle.sk_f64(S1, S2, M)
    for f in range(20):
        s1, s2 = int(S1[f, 0]), int(S2[f, 0])
        exact = (M + 1) / (M - 1) * (M * s2 / (s1 * s1) - 1)
        assert abs(sk64[f] - exact) <= 1e-12 * abs(exact)
    single = oracle.sk_single_f64(S1, S2, M)[:, 0]
    assert np.allclose(single, sk64, rtol=1e-13, atol=0)


def test_scale_invariance_bit_exact():
    """Overall scaling of an input leaves SK unchanged (Sec. 2: scaling-invariant probe)."""
    rng = np.random.default_rng(5)
    M, N = 256, 32
    re = rng.integers(-3, 4, size=(4, M, N))
    im = rng.integers(-3, 4, size=(4, M, N))
    x1 = _pack(re, im).reshape(4, M * N)
    scale = np.where(np.arange(N) % 2 == 0, 2, 1)      # double every other input
    x2 = _pack(re * scale, im * scale).reshape(4, M * N)
    a = oracle.flag(x1, M, N)
    b = oracle.flag(x2, M, N)
    assert (a["Q"] == b["Q"]).all() and (a["sk"] == b["sk"]).all()
    assert np.allclose(a["sk64"], b["sk64"], rtol=1e-14, atol=0)


def test_permutation_invariance():
    rng = np.random.default_rng(9)
    M, N = 128, 24
    x = _random_bytes(rng, 3, M, N).reshape(3, M, N)
    a = oracle.flag(x.reshape(3, -1), M, N)
    xp = x[:, rng.permutation(M), :][:, :, rng.permutation(N)]
    b = oracle.flag(np.ascontiguousarray(xp).reshape(3, -1), M, N)
    assert (a["Q"] == b["Q"]).all() and (a["neff"] == b["neff"]).all()


def test_dead_inputs_are_excluded():
    rng = np.random.default_rng(4)
    M, N = 32, 6
    x = _random_bytes(rng, 2, M, N).reshape(2, M, N)
    x[:, :, 2] = 0x88          # input 2 has no power
    x[1, :, :] = 0x88          # frame 1: no input has power
    r = oracle.flag(x.reshape(2, -1), M, N)
    assert r["neff"][0] == N - 1 and r["neff"][1] == 0
    assert np.isnan(r["sk"][1]) and r["mask"][1] == 1
    keep = [0, 1, 3, 4, 5]
    y = np.ascontiguousarray(x[:1, :, keep]).reshape(1, -1)
    s = oracle.flag(y, M, 5)
    assert s["Q"][0] == r["Q"][0]


# --------------------------------------------------------------------------
# moments under complex Gaussian input (Sec. 2.1 and Eq. final moments)
# --------------------------------------------------------------------------

def _cgauss(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("M,N", [(256, 16), (64, 64)])
def test_mean_one_and_variance_4_over_nN(M, N):
    rng = np.random.default_rng(100 + M + N)
    T = 3000
    sk = np.concatenate([oracle.sk_from_complex(_cgauss(rng, (500, M, N))) for _ in range(T // 500)])
    var_pred = 4.0 / (M * N)
    # mean exactly 1 for the unbiased estimator; 5 standard errors
    assert abs(sk.mean() - 1.0) < 5 * math.sqrt(var_pred / T)
    # first-order variance 4/(nN), O(1/(n^2 N)) correction plus sampling error (~2.6 %)
    assert abs(sk.var() / var_pred - 1.0) < 0.10


def test_single_receiver_skew_and_kurtosis():
    """skew ~ 10/sqrt(n), kurtosis ~ 246/n for SK^ (Sec. 2.1), at n = 512."""
    rng = np.random.default_rng(77)
    M = 512
    vals = np.concatenate([oracle.sk_from_complex(_cgauss(rng, (2000, M, 1))) for _ in range(40)])
    z = (vals - vals.mean()) / vals.std()
    skew = (z ** 3).mean()
    kurt = (z ** 4).mean() - 3.0
    assert abs(skew / (10 / math.sqrt(M)) - 1) < 0.15
    assert abs(kurt / (246 / M) - 1) < 0.35
    assert abs(vals.var() / (4 / M) - 1) < 0.05


def test_combination_keeps_statistics_of_average():
    """SK~ = Avg(SK^_i) (Eq. final): variance falls as 1/N at fixed n."""
    rng = np.random.default_rng(31)
    M = 128
    v1 = oracle.sk_from_complex(_cgauss(rng, (4000, M, 1))).var()
    v16 = oracle.sk_from_complex(_cgauss(rng, (4000, M, 16))).var()
    assert abs((v1 / v16) / 16 - 1) < 0.12


# --------------------------------------------------------------------------
# App. B digitisation model
# --------------------------------------------------------------------------

@pytest.mark.parametrize("s", [1.4, 1.52, 2.5])
def test_sheppard_corrections_unclipped(s):
    """Rounding to integers: m2 = s^2 + 1/12, m4 = 3 s^4 + s^2/2 + 1/80 (Sheppard).

    Exact up to terms of order exp(-2 pi^2 s^2), below 1e-12 for s >= 1.4.
    """
    m2, m4 = dg.moments(s, lim=None)
    assert abs(m2 - (s * s + 1 / 12)) < 1e-12
    assert abs(m4 - (3 * s ** 4 + s * s / 2 + 1 / 80)) < 1e-10


def test_digitisation_limits():
    # CHIME-like rms 1.52 LSB gives a small negative offset ("slightly offset", Fig. skdists)
    d = float(dg.delta_of_sigma(1.52))
    assert -2e-3 < d < 0
    # very large sigma: every component is +-7, |x|^2 = 98 constant, SK^ = 0, delta = -1
    assert abs(float(dg.delta_of_sigma(1e4)) + 1.0) < 1e-3
    # an unclipped continuous Gaussian has no offset: the clipped model tends to Sheppard's
    m2, m4 = dg.moments(1.52, lim=None)
    assert abs(float(dg.delta_of_sigma(1.52, lim=None)) - (m4 / (2 * m2 * m2) - 1.5)) < 1e-15
    # inverse power map recovers sigma
    for s in (1.5, 2.0, 3.3):
        m2, _ = dg.moments(s)
        assert abs(float(dg.sigma_of_power(2 * m2)[0]) - s) < 1e-9


@pytest.mark.slow
def test_digitised_mean_offset_monte_carlo():
    """Quantised Gaussian data: mean(SK~) - 1 converges to delta(sigma) (App. B)."""
    import synth

    M, N = 256, 64
    for sigma in (1.52, 2.5, 3.0):
        ds = synth.Dataset(n_frames=400, M=M, N=N, seed=synth.sub_seed(90, int(sigma * 100)),
                           sigma=np.full(N, sigma))
        x = ds.generate_cpu()
        r = oracle.flag(x, M, N)
        se = math.sqrt(4.0 / (M * N) / 400)
        d = float(dg.delta_of_sigma(sigma))
        # model is the large-n limit; allow 5 standard errors plus an O(1/n) term
        assert abs(r["sk64"].mean() - 1.0 - d) < 5 * se + 0.5 / M


# --------------------------------------------------------------------------
# thresholds (Sec. 3.2)
# --------------------------------------------------------------------------

def test_thresholds_bracket_centre_symmetrically():
    M, N = 256, 64
    lo, hi = oracle.thresholds(M, N, 3.0, -0.01)
    for ne in (1, 7, 64):
        c = (1 - 0.01) * (M - 1) * ne * 2 ** 32 / (M + 1)
        w = 3.0 * 2 / math.sqrt(M * ne) * (M - 1) * ne * 2 ** 32 / (M + 1)
        assert abs(hi[ne] - (c + w)) <= 1 + 1e-15 * c
        assert abs(lo[ne] - (c - w)) <= 1 + 1e-15 * c
        assert hi[ne] - c == pytest.approx(c - lo[ne], rel=1e-9)


def test_mask_agrees_with_exact_interval():
    """Integer recipe = 'outside mean +- a sqrt(var)' on the exact SK~, except at fp32 ties."""
    rng = np.random.default_rng(21)
    M, N = 16, 8
    x = _random_bytes(rng, 60, M, N)
    r = oracle.flag(x, M, N, n_sigma=1.0, mean_offset=0.3)
    flips = 0
    for f in range(60):
        bs1, bs2 = brute.sums(list(x[f]), M, N)
        sk, _, _, ne = brute.sk_normalised(bs1, bs2, M)
        want = 1 if ne == 0 else brute.outside(sk, M, ne, 1.0, 0.3)
        if want != r["mask"][f]:
            flips += 1
            # only allowed when SK~ is within fp32 rounding of an edge
            half = 2 / math.sqrt(M * ne)
            edge = min(abs(float(sk) - 1.3 - half), abs(float(sk) - 1.3 + half))
            assert edge < 1e-5
    assert flips <= 1


@pytest.mark.slow
def test_false_alarm_rate_at_three_sigma():
    """Clean Gaussian data, large nN: about 0.27 % of frames outside +-3 sigma (Sec. 3.2)."""
    rng = np.random.default_rng(123)
    M, N = 256, 64
    n_flag = 0
    T = 0
    for _ in range(8):
        sk = oracle.sk_from_complex(_cgauss(rng, (1000, M, N)))
        half = 3 * 2 / math.sqrt(M * N)
        n_flag += int(((sk > 1 + half) | (sk < 1 - half)).sum())
        T += 1000
    assert 0.0008 < n_flag / T < 0.0065


def test_independent_estimates_against_exact_rationals():
    """Per-input SK^_i (Eq. originalSK) and its one-input flag (Sec. 2.2.3 independent
    estimates); their average is SK~ (Eq. final, third line)."""
    rng = np.random.default_rng(44)
    M, N = 16, 6
    x = _random_bytes(rng, 12, M, N)
    x[3, :N] = 0x88   # make a few inputs dead in frame 3 (t = 0 row only: still powered)
    r = oracle.flag_inputs(x, M, N, n_sigma=1.0, mean_offset=0.2)
    full = oracle.flag(x, M, N)
    for f in range(12):
        bs1, bs2 = brute.sums(list(x[f]), M, N)
        vals = []
        for i in range(N):
            if bs1[i] == 0:
                assert r["valid"][f, i] == 0 and np.isnan(r["sk_in"][f, i])
                assert r["mask_in"][f, i] == 1
                continue
            e = brute.sk_single(bs1[i], bs2[i], M)
            vals.append(e)
            assert abs(float(r["sk_in"][f, i]) - float(e)) <= 1e-6 * abs(float(e)) + 1e-9
            want = brute.outside(e, M, 1, 1.0, 0.2)
            edge = min(abs(float(e) - 1.2 - 2 / math.sqrt(M)), abs(float(e) - 1.2 + 2 / math.sqrt(M)))
            assert r["mask_in"][f, i] == want or edge < 1e-5
        if vals:
            avg = sum(vals, Fraction(0)) / len(vals)
            assert abs(float(avg) - full["sk64"][f]) <= 1e-12 * max(1, abs(float(avg)))


def test_pearson3_thresholds_limits():
    """Large m: the Pearson III edges tend to the symmetric +-a sigma interval, their
    offset shrinking like the skewness, 1/sqrt(m)."""
    M, N = 256, 4096
    slo, shi = oracle.thresholds(M, N, 3.0, 0.01)
    plo, phi = oracle.thresholds(M, N, 3.0, 0.01, pearson3=True)

    def rel(ne):
        half = (shi[ne] - slo[ne]) / 2
        return (phi[ne] - shi[ne]) / half, (plo[ne] - slo[ne]) / half

    hi_n, lo_n = rel(N)
    hi_q, lo_q = rel(N // 4)
    assert 0 < hi_n < 0.01 and 0 < lo_n < 0.01
    assert abs(hi_q / hi_n - 2.0) < 0.05 and abs(lo_q / lo_n - 2.0) < 0.05
    # skewed to the right at small m: both edges above the symmetric ones
    assert phi[1] > shi[1] and plo[1] > slo[1]


@pytest.mark.slow
def test_pearson3_false_alarm_balance():
    """Small nN (Sec. 3.2): the skewed thresholds balance the two tails, which the
    symmetric interval does not.  Complex Gaussian input, a = 2 (p = 2.28 % per tail)."""
    from scipy.stats import norm

    rng = np.random.default_rng(2018)
    M, N, a = 128, 2, 2.0
    p = norm.sf(a)
    sk = np.concatenate([oracle.sk_from_complex(_cgauss(rng, (20000, M, N))) for _ in range(8)])
    m = M * N
    slo, shi = 1 - a * 2 / math.sqrt(m), 1 + a * 2 / math.sqrt(m)
    k = m / 25.0
    phi = 0.6 + 0.4 * (1 - 1 / (9 * k) + a / (3 * math.sqrt(k))) ** 3
    plo = 0.6 + 0.4 * (1 - 1 / (9 * k) - a / (3 * math.sqrt(k))) ** 3
    # the oracle's integer thresholds encode these edges
    tlo, thi = oracle.thresholds(M, 1, a, 0.0, pearson3=True)
    scale = (M - 1) * 2 ** 32 / (M + 1)
    assert abs(thi[1] / scale - (0.6 + 0.4 * (1 - 1 / (9 * M / 25) + a / (3 * math.sqrt(M / 25))) ** 3)) < 1e-9
    up_s, lo_s = (sk > shi).mean(), (sk < slo).mean()
    up_p, lo_p = (sk > phi).mean(), (sk < plo).mean()
    assert up_s > 1.3 * p and lo_s < 0.5 * p                 # symmetric: unbalanced
    assert 0.7 * p < up_p < 1.4 * p and 0.7 * p < lo_p < 1.4 * p


def test_pearson3_matches_exact_gamma_quantile():
    """The Pearson III thresholds against the exact quantiles of the same shifted gamma
    (shape m/25, scale 10/m, mean 1+delta) from scipy: the Wilson-Hilferty form the
    oracle uses is within 1 % of the distance from the centre at m = M N_eff >= 256,
    and its error shrinks as m grows."""
    from scipy import stats

    delta = -0.02
    for a in (2.0, 3.0):
        errs = []
        for M, ne in ((256, 1), (128, 8), (256, 16), (256, 64)):
            m = M * ne
            t_lo, t_hi = oracle.thresholds(M, ne, a, delta, pearson3=True)
            f = (M + 1) / ((M - 1) * ne * 2.0 ** 32)
            k, scale, loc = m / 25.0, 10.0 / m, 1.0 + delta - 0.4
            for t, p in ((t_hi[ne], stats.norm.cdf(a)), (t_lo[ne], stats.norm.cdf(-a))):
                exact = loc + stats.gamma.ppf(p, k, scale=scale)
                err = abs(t * f - exact) / abs(exact - (1.0 + delta))
                assert err < 0.01, (a, M, ne, err)
                errs.append((m, err))
        by_m = {}
        for m, e in errs:
            by_m[m] = max(by_m.get(m, 0.0), e)
        ms = sorted(by_m)
        assert all(by_m[x] >= by_m[y] for x, y in zip(ms, ms[1:]))
