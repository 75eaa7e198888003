"""ORACLE -- test infrastructure only.

A plain, slow CPU statement of the multi-receiver spectral-kurtosis RFI
detector of Taylor et al., "Spectral Kurtosis Based RFI Mitigation for CHIME"
(arXiv:1808.10365).  Only `tests/`, `__graft_entry__.smoke()` and the CPU
baseline and reference-arm legs of `bench.py` may import it.  It shares no code with the CUDA
library and never calls it; its inputs come from the `synth` generator or
from the tests themselves.

Notation: M samples per input per estimate (the paper's n), N inputs (the
paper's N), N_eff the inputs with non-zero power.

Pieces and the passages they follow (every function cites its own):
  * `power_sums`         Eq. 1 / Eq. (singlesums)            [sk_oracle.c]
  * `sk_f64`             Eqs. (discreteMean)-(normedSum2), (final)  fp64
  * `sk_spec`            Eq. (final) via Avg(SK^_i) in the CUDA path's declared
                         precision (int64 D_i, one fp32 divide, 2^32 fixed
                         point sum) so Q and masks compare bit for bit
  * `thresholds`, `mask` Sec. 3.2: flag outside mean +- a*sqrt(var), with
                         var = 4/(n N) (Eq. final moments) and the mean shifted
                         by the digitisation offset (App. B); `pearson3`: the
                         false-alarm (shifted gamma) thresholds for small n N
  * `flag_inputs`        Eq. (originalSK) per input (independent estimates)
  * `digitisation`       App. B: mean offset of SK for clipped 4-bit data
  * `served_flags`       running per-input power state feeding the App. B offset,
                         and the running-mu form of Eq. (avgSK)
  * `brute`              exact rational arithmetic on tiny inputs

Parity status: S1, S2, Q, N_eff, SK and the static mask are pinned (closed
forms, brute force, moments; tests/test_oracle_pins.py).  The Pearson III
thresholds are pinned against exact gamma quantiles, the served state by its
fixed point and a power step.  The integer threshold recipe and the
digitisation-offset table are pinned only by Monte-Carlo false-alarm rates and
by limits of the model (the paper prints no threshold numbers): parity for
those is "partial" in the strict sense.
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")
TWO32 = 4294967296.0

_lib = None


def build():
    """Compile the C part of the oracle (plain gcc, no FMA contraction)."""
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-fno-fast-math", "-std=c11", "-o", LIB,
                    os.path.join(HERE, "sk_oracle.c"), "-lm"], check=True)


def _load():
    global _lib
    if _lib is None:
        src = os.path.join(HERE, "sk_oracle.c")
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(src):
            build()
        lib = ctypes.CDLL(LIB)
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        lib.oracle_power_sums.argtypes = [P, i64, i32, i32, i32, P, P]
        lib.oracle_sk_f64.argtypes = [P, P, i64, i32, i32, P, P, P]
        lib.oracle_sk_spec.argtypes = [P, P, i64, i32, i32, P, P, P]
        lib.oracle_sk_single_f64.argtypes = [P, P, i64, i32, P]
        lib.oracle_terms_spec.argtypes = [P, P, i64, i32, P, P, P]
        lib.oracle_max_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(_load().oracle_max_threads())


def set_threads(n: int) -> None:
    """Threads the oracle's C loops use from now on (timing only)."""
    _load().oracle_set_threads(int(n))


def power_sums(x: np.ndarray, M: int, N: int, layout: int = 0):
    """S1, S2 (int64 [frames, N]) of Eq. 1 for bytes x ([frames, M*N] uint8)."""
    x = np.ascontiguousarray(x, dtype=np.uint8).reshape(-1, M * N)
    F = x.shape[0]
    S1 = np.zeros((F, N), dtype=np.int64)
    S2 = np.zeros((F, N), dtype=np.int64)
    _load().oracle_power_sums(_p(x), F, M, N, layout, _p(S1), _p(S2))
    return S1, S2


def sk_f64(S1: np.ndarray, S2: np.ndarray, M: int):
    """(SK~ fp64, S1bar, N_eff) per frame from Eqs. discreteMean..final in fp64."""
    S1 = np.ascontiguousarray(S1, dtype=np.int64)
    S2 = np.ascontiguousarray(S2, dtype=np.int64)
    F, N = S1.shape
    sk = np.zeros(F, dtype=np.float64)
    sb1 = np.zeros(F, dtype=np.float64)
    ne = np.zeros(F, dtype=np.int32)
    _load().oracle_sk_f64(_p(S1), _p(S2), F, M, N, _p(sk), _p(sb1), _p(ne))
    return sk, sb1, ne


def sk_spec(S1: np.ndarray, S2: np.ndarray, M: int):
    """(Q int64, N_eff int32, SK~ fp32) per frame in the CUDA path's declared precision."""
    S1 = np.ascontiguousarray(S1, dtype=np.int64)
    S2 = np.ascontiguousarray(S2, dtype=np.int64)
    F, N = S1.shape
    Q = np.zeros(F, dtype=np.int64)
    ne = np.zeros(F, dtype=np.int32)
    sk = np.zeros(F, dtype=np.float32)
    _load().oracle_sk_spec(_p(S1), _p(S2), F, M, N, _p(Q), _p(ne), _p(sk))
    return Q, ne, sk


def sk_single_f64(S1: np.ndarray, S2: np.ndarray, M: int) -> np.ndarray:
    """Per-input SK^_i (Eq. originalSK) in fp64, NaN where S1_i = 0."""
    S1 = np.ascontiguousarray(S1, dtype=np.int64)
    S2 = np.ascontiguousarray(S2, dtype=np.int64)
    out = np.zeros(S1.shape, dtype=np.float64)
    _load().oracle_sk_single_f64(_p(S1), _p(S2), S1.size, M, _p(out))
    return out


def terms_spec(S1: np.ndarray, S2: np.ndarray, M: int):
    """Per-input (q_i, SK^_i fp32, valid) in the kernel precision (Eq. originalSK)."""
    S1 = np.ascontiguousarray(S1, dtype=np.int64)
    S2 = np.ascontiguousarray(S2, dtype=np.int64)
    q = np.zeros(S1.shape, dtype=np.int64)
    sk1 = np.zeros(S1.shape, dtype=np.float32)
    valid = np.zeros(S1.shape, dtype=np.uint8)
    _load().oracle_terms_spec(_p(S1), _p(S2), S1.size, M, _p(q), _p(sk1), _p(valid))
    return q, sk1, valid


def flag_inputs(x: np.ndarray, M: int, N: int, n_sigma: float = 3.0, mean_offset: float = 0.0,
                layout: int = 0):
    """Independent single-receiver estimates and flags (Sec. 2.2.3, Eq. originalSK):
    each input tested alone against the one-input interval (N_eff = 1 thresholds)."""
    S1, S2 = power_sums(x, M, N, layout)
    q, sk1, valid = terms_spec(S1, S2, M)
    t_lo, t_hi = thresholds(M, 1, n_sigma, mean_offset)
    m = ((q > t_hi[1]) | (q < t_lo[1]) | (valid == 0)).astype(np.uint8)
    return dict(sk_in=sk1, mask_in=m, sk_in64=sk_single_f64(S1, S2, M), valid=valid)


def sk_from_complex(x: np.ndarray) -> np.ndarray:
    """SK~ per frame for float complex samples x [frames, M, N] (the non-digitised path of App. B).

    Follows Eqs. (singlesums), (discreteMean), (normedSum2), (final) in fp64.
    """
    p = (x.real ** 2 + x.imag ** 2)
    M = x.shape[1]
    N = x.shape[2]
    S1 = p.sum(axis=1)
    S2 = (p * p).sum(axis=1)
    mu = S1 / M
    s2bar = (S2 / (mu * mu)).sum(axis=1)
    return (M + 1.0) / (M - 1.0) * (s2bar / (M * N) - 1.0)


# ----------------------------------------------------------------------------
# thresholds and mask (Sec. 3.2, Eq. final moments, App. B)
# ----------------------------------------------------------------------------

def thresholds(M: int, N: int, n_sigma: float, mean_offset: float = 0.0,
               pearson3: bool = False):
    """Integer thresholds on Q for N_eff = 0..N (entry 0 unused).

    The centre is mean(SK~) = 1 (Eq. final moments) plus the digitisation offset
    delta (App. B); the half-width a*sqrt(var) with var = 4/(n N_eff).  In Q units
    SK~ = (n+1)/((n-1) N_eff) * Q / 2^32, so SK~ > X  <=>  Q > X (n-1) N_eff 2^32/(n+1).
    Evaluated in double in exactly this order:
      X_hi = ((1+delta) + a*s) * (n-1) * N_eff * 2^32 / (n+1),  T_hi = floor(X_hi)
      X_lo = ((1+delta) - a*s) * (n-1) * N_eff * 2^32 / (n+1),  T_lo = ceil(X_lo)
    with s = 2 / sqrt(n * N_eff).

    pearson3: false-alarm thresholds for small m = n N_eff (Sec. 3.2).  SK~ is
    taken as a Pearson type III (shifted gamma) with mean 1+delta, variance 4/m
    and skewness 10/sqrt(m) (Sec. 2.1 moments averaged over N_eff inputs), i.e.
    shape k = m/25, scale 10/m, location (1+delta) - 0.4; each threshold is its
    gamma quantile at normal deviate +-a by Wilson-Hilferty,
    k (1 - 1/(9k) + z/(3 sqrt(k)))^3.
    """
    t_lo = np.zeros(N + 1, dtype=np.int64)
    t_hi = np.zeros(N + 1, dtype=np.int64)
    centre = 1.0 + float(mean_offset)
    a = float(n_sigma)
    for ne in range(1, N + 1):
        m = float(M * ne)
        if pearson3:
            k = m / 25.0
            b_hi = 1.0 - 1.0 / (9.0 * k) + a / (3.0 * math.sqrt(k))
            b_lo = 1.0 - 1.0 / (9.0 * k) - a / (3.0 * math.sqrt(k))
            v_hi = (centre - 0.4) + 0.4 * (b_hi * b_hi * b_hi)
            v_lo = (centre - 0.4) + 0.4 * (b_lo * b_lo * b_lo)
        else:
            s = 2.0 / math.sqrt(m)
            v_hi = centre + a * s
            v_lo = centre - a * s
        x_hi = v_hi * float(M - 1) * float(ne) * TWO32 / float(M + 1)
        x_lo = v_lo * float(M - 1) * float(ne) * TWO32 / float(M + 1)
        t_hi[ne] = math.floor(x_hi)
        t_lo[ne] = math.ceil(x_lo)
    return t_lo, t_hi


def mask(Q: np.ndarray, neff: np.ndarray, t_lo: np.ndarray, t_hi: np.ndarray,
         shift: np.ndarray | None = None) -> np.ndarray:
    """1 where SK~ lies strictly outside [lo, hi] or no input had power (Sec. 3.2)."""
    ne = np.asarray(neff, dtype=np.int64)
    lo = t_lo[ne].copy()
    hi = t_hi[ne].copy()
    if shift is not None:
        lo = lo + shift
        hi = hi + shift
    m = (Q > hi) | (Q < lo) | (ne == 0)
    return m.astype(np.uint8)


def flag(x: np.ndarray, M: int, N: int, n_sigma: float = 3.0, mean_offset: float = 0.0,
         layout: int = 0, pearson3: bool = False):
    """Whole plain path on bytes x: dict with S1, S2, Q, neff, sk (fp32), mask, sk64."""
    S1, S2 = power_sums(x, M, N, layout)
    Q, ne, sk = sk_spec(S1, S2, M)
    sk64, _, _ = sk_f64(S1, S2, M)
    t_lo, t_hi = thresholds(M, N, n_sigma, mean_offset, pearson3)
    return dict(S1=S1, S2=S2, Q=Q, neff=ne, sk=sk, sk64=sk64,
                mask=mask(Q, ne, t_lo, t_hi), t_lo=t_lo, t_hi=t_hi)


from . import digitisation  # noqa: E402
from .served import served_flags  # noqa: E402,F401
