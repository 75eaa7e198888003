"""ORACLE (test infrastructure only): the served path's running power state.

Per stream, frames in arrival order.  Each input i keeps an integer power
state P_i (a leaky integrator of S1_i with gain 2^-k) that estimates its mean
power; the App. B digitisation offset delta(P_i) of each input then shifts the
flagging thresholds, so the centre follows each input's own level instead of
one static offset (the paper adds the simulated offset to the threshold,
App. B).  Flagged frames leave the state unchanged, so RFI does not drag it.

  first frame of a stream:   P_i = S1_i << k
  bucket(P) = min(B - 1, floor(P B / (2^k n 128)))
  E = sum over inputs with S1_i > 0 of e[bucket(P_i)]
  mask = Q > T_hi[N_eff] + E  or  Q < T_lo[N_eff] + E  or  N_eff = 0
  if mask == 0:  P_i <- P_i - (P_i >> k) + S1_i     (every input)
e[] is the digitisation offset table (oracle.digitisation.offset_table).

Running-mu variant (running_mu=True): each input is normalised by its running
power per sample mu_i = P_i / (2^k n) instead of the frame's own S1_i / n, and
the combined estimator takes the general form of Eq. (avgSK), first line, with
n' = n N_eff, S1bar = sum S1_i/mu_i, S2bar = sum S2_i/mu_i^2, rescaled to SK~ by
Eq. (final), first line.  In the precision the CUDA path declares, per input
  a_i = fp32(S1_i 2^k n) / fp32(P_i),  b_i = fp32(S2_i (2^k n)^2) / fp32(P_i^2)
(integer numerators and denominators exact, one fp32 divide each), summed as
A = sum rint(2^24 a_i), B = sum rint(2^24 b_i) in int64, and then in IEEE double
  sk_hat = (n'+1)/(n'-1) * (n' B 2^-24 / (A 2^-24)^2 - 1)
  sk     = (n'-1)(n+1) / ((n'+1)(n-1)) * sk_hat
flagged outside [lo, hi] of the symmetric interval (centre 1 + delta_state,
half-width a 2/sqrt(n'), delta_state = E (n+1) / ((n-1) N_eff 2^32)), every
operation in that order.
"""

from __future__ import annotations

import math

import numpy as np

from . import power_sums, sk_spec, thresholds


def bucket(P: np.ndarray, M: int, B: int = 4096, k: int = 6) -> np.ndarray:
    b = (P.astype(np.uint64) * np.uint64(B)) // np.uint64((1 << k) * M * 128)
    return np.minimum(b, np.uint64(B - 1)).astype(np.int64)


def f32_of_int(x: int) -> np.float32:
    """Nearest fp32 to the integer x, ties to even, rounded once (exact integer work)."""
    if x == 0:
        return np.float32(0.0)
    neg = x < 0
    v = -x if neg else x
    nb = v.bit_length()
    if nb <= 24:
        r = np.float32(v)
    else:
        sh = nb - 24
        m, rem = v >> sh, v & ((1 << sh) - 1)
        half = 1 << (sh - 1)
        if rem > half or (rem == half and (m & 1)):
            m += 1
        r = np.float32(float(m) * 2.0 ** sh)   # m <= 2^24: exact in double and fp32
    return np.float32(-r) if neg else r


def _running_mu_sk(S1, S2, P, M, k):
    """(A, B, N_eff, sk_double) of the running-mu estimator for one frame."""
    A = 0
    Bq = 0
    ne = 0
    sc = (1 << k) * M
    for s1, s2, p in zip(S1.tolist(), S2.tolist(), P.tolist()):
        if s1 <= 0 or p <= 0:
            continue
        a = np.float32(f32_of_int(s1 * sc) / f32_of_int(p))
        b = np.float32(f32_of_int(s2 * sc * sc) / f32_of_int(p * p))
        A += int(np.rint(np.float64(a) * 16777216.0))
        Bq += int(np.rint(np.float64(b) * 16777216.0))
        ne += 1
    if ne == 0 or A == 0:
        return A, Bq, ne, float("nan")
    m = float(M * ne)
    a_f = float(A) * (2.0 ** -24)
    b_f = float(Bq) * (2.0 ** -24)
    sk_hat = (m + 1.0) / (m - 1.0) * (m * b_f / (a_f * a_f) - 1.0)
    sk = (m - 1.0) * float(M + 1) / ((m + 1.0) * float(M - 1)) * sk_hat
    return A, Bq, ne, sk


def served_flags(frames: np.ndarray, M: int, N: int, e: np.ndarray, n_sigma: float = 3.0,
                 mean_offset: float = 0.0, k: int = 6, B: int = 4096, layout: int = 0,
                 P0: np.ndarray | None = None, running_mu: bool = False):
    """Run one stream's frames ([T, M*N] uint8) in order.

    Returns dict(Q, neff, sk, mask, E, P) with P the state after the last frame.
    P0 continues from an earlier state (checkpoint); None starts a new stream.
    """
    frames = np.asarray(frames, dtype=np.uint8).reshape(-1, M * N)
    T = frames.shape[0]
    t_lo, t_hi = thresholds(M, N, n_sigma, mean_offset)
    S1, S2 = power_sums(frames, M, N, layout)
    Q, ne, sk = sk_spec(S1, S2, M)
    P = None if P0 is None else np.asarray(P0, dtype=np.int64).copy()
    msk = np.zeros(T, dtype=np.uint8)
    E = np.zeros(T, dtype=np.int64)
    sk_out = sk.copy()
    for f in range(T):
        s1 = S1[f]
        if P is None:
            P = s1 << k
        valid = s1 > 0
        E[f] = int(e[bucket(P, M, B, k)][valid].sum())
        n = int(ne[f])
        if running_mu:
            _, _, nr, skd = _running_mu_sk(s1, S2[f], P, M, k)
            if nr == 0 or skd != skd:
                m = True
            else:
                mp = float(M * nr)
                centre = 1.0 + float(mean_offset) + float(E[f]) * float(M + 1) / (
                    float(M - 1) * float(nr) * 4294967296.0)
                half = float(n_sigma) * 2.0 / math.sqrt(mp)
                m = skd > centre + half or skd < centre - half
            sk_out[f] = np.float32(skd)
        else:
            m = (n == 0) or (Q[f] > t_hi[n] + E[f]) or (Q[f] < t_lo[n] + E[f])
        msk[f] = 1 if m else 0
        if not m:
            P = P - (P >> k) + s1
    return dict(Q=Q, neff=ne, sk=sk_out, mask=msk, E=E, P=P, S1=S1, S2=S2)
