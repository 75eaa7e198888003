"""ORACLE (test infrastructure only): exact rational arithmetic for tiny inputs.

Pure-Python loops over Fractions; every formula is written as the paper
prints it, so these serve as the brute-force pins for the C oracle.
"""

from __future__ import annotations

from decimal import Decimal, getcontext
from fractions import Fraction


def unpack(b: int):
    """4+4-bit offset binary: (real, imag) = (high nibble - 8, low nibble - 8)."""
    return (b >> 4) - 8, (b & 15) - 8


def sums(frame, M: int, N: int, layout: int = 0):
    """S1_i, S2_i (Eq. singlesums) for one frame given as a flat sequence of M*N bytes."""
    S1 = [0] * N
    S2 = [0] * N
    for i in range(N):
        for t in range(M):
            b = frame[t * N + i] if layout == 0 else frame[i * M + t]
            re, im = unpack(int(b))
            p = re * re + im * im
            S1[i] += p
            S2[i] += p * p
    return S1, S2


def sk_single(s1: int, s2: int, n: int) -> Fraction:
    """SK^_i of one receiver, Eq. (originalSK)."""
    return Fraction(n + 1, n - 1) * (Fraction(n * s2, s1 * s1) - 1)


def sk_normalised(S1, S2, n: int):
    """SK~ from the normalised cumulants, Eqs. (discreteMean), (normedSum2), (final) 2nd line.

    Returns (SK~, S1bar, S2bar, N_eff); inputs with S1_i = 0 are left out.
    """
    s1bar = Fraction(0)
    s2bar = Fraction(0)
    ne = 0
    for s1, s2 in zip(S1, S2):
        if s1 == 0:
            continue
        mu = Fraction(s1, n)
        s1bar += Fraction(s1) / mu
        s2bar += Fraction(s2) / (mu * mu)
        ne += 1
    if ne == 0:
        return None, s1bar, s2bar, 0
    sk = Fraction(n + 1, n - 1) * (s2bar / (n * ne) - 1)
    return sk, s1bar, s2bar, ne


def sk_average(S1, S2, n: int):
    """SK~ = Avg(SK^_i), Eq. (final) 3rd line."""
    vals = [sk_single(s1, s2, n) for s1, s2 in zip(S1, S2) if s1 != 0]
    if not vals:
        return None
    return sum(vals, Fraction(0)) / len(vals)


def sk_combined_hat(S1, S2, n: int):
    """Unscaled multi-receiver SK^ over M' = nN samples, Eq. (avgSK) 1st line."""
    sk, s1bar, s2bar, ne = sk_normalised(S1, S2, n)
    if ne == 0:
        return None
    Mp = n * ne
    return Fraction(Mp + 1, Mp - 1) * (Mp * s2bar / (s1bar * s1bar) - 1)


def rescale_hat(sk_hat: Fraction, n: int, N: int) -> Fraction:
    """SK~ from SK^, Eq. (final) 1st line."""
    return Fraction((n * N - 1) * (n + 1), (n * N + 1) * (n - 1)) * sk_hat


def outside(sk: Fraction, n: int, ne: int, n_sigma: float, mean_offset: float = 0.0) -> int:
    """1 if SK~ lies strictly outside (1+delta) +- a*2/sqrt(n N_eff) (Sec. 3.2), at 60 digits."""
    getcontext().prec = 60
    centre = Decimal(1) + Decimal(mean_offset)
    half = Decimal(n_sigma) * Decimal(2) / (Decimal(n * ne).sqrt())
    v = Decimal(sk.numerator) / Decimal(sk.denominator)
    return 1 if (v > centre + half or v < centre - half) else 0


def sk_running_mu(S1, S2, mu, n: int):
    """SK~ with each receiver normalised by a given mean power per sample mu_i
    instead of its frame's own S1_i/n (the running-mu reading of the served path).

    Eq. (avgSK) 1st line over M' = n N_eff samples, with S1bar = sum S1_i/mu_i and
    S2bar = sum S2_i/mu_i^2 (Eq. normedSum1/normedSum2 with mu_i given), then
    rescaled to SK~ by Eq. (final) 1st line.  Receivers with S1_i = 0 or mu_i = 0
    are left out.  Returns (SK~ as a Fraction or None, N_eff, n' S2bar / S1bar^2).
    """
    s1bar = Fraction(0)
    s2bar = Fraction(0)
    ne = 0
    for s1, s2, m in zip(S1, S2, mu):
        m = Fraction(m)
        if s1 == 0 or m == 0:
            continue
        s1bar += Fraction(s1) / m
        s2bar += Fraction(s2) / (m * m)
        ne += 1
    if ne == 0:
        return None, 0, None
    Mp = n * ne
    ratio = Mp * s2bar / (s1bar * s1bar)
    sk_hat = Fraction(Mp + 1, Mp - 1) * (ratio - 1)
    return rescale_hat(sk_hat, n, ne), ne, ratio
