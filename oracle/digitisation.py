"""ORACLE (test infrastructure only): digitisation offset of SK~ (paper App. B).

The paper shifts the flagging threshold's centre by the mean offset of SK~
that 4+4-bit quantisation (values clipped to [-7, 7]) produces, obtained from
a simulation of the correlator's data characteristics (App. B).  This module
states that offset as a model instead of a simulation:

  a component is v = clip(round(sigma g), -L, L), g ~ N(0, 1), L = 7;
  m2 = E[v^2], m4 = E[v^4] from the exact level probabilities;
  for x = v_re + i v_im (independent parts): E|x|^2 = 2 m2,
  E|x|^4 = 2 m4 + 2 m2^2, and for large n SK^ -> E|x|^4 / (E|x|^2)^2 - 1, so
  delta(sigma) = m4 / (2 m2^2) - 3/2     (0 for an unquantised Gaussian).

For the running per-input state, a mean power per sample mu = E|x|^2 is
mapped back to sigma by solving 2 m2(sigma) = mu (bisection; m2 rises with
sigma), giving delta(mu).

The model is pinned by Sheppard's corrections (no clipping), by its
large-sigma limit (two-level +-L data: SK^ = 0, delta = -1) and by Monte Carlo
on generated data (tests/test_oracle_pins.py).
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

SQRT2 = math.sqrt(2.0)


def level_probs(sigma, lim: int | None = 7):
    """P(v = k) for k = -K..K (K = lim, or wide enough when unclipped), shape [..., 2K+1]."""
    sigma = np.asarray(sigma, dtype=np.float64)[..., None]
    if lim is None:
        K = int(np.ceil(40.0 * float(np.max(sigma)) + 10.0))
    else:
        K = int(lim)
    # v >= 0 from upper tails (accurate far out), v < 0 by symmetry of g
    kp = np.arange(0, K + 1, dtype=np.float64)
    up_lo = 0.5 * erfc((kp - 0.5) / (sigma * SQRT2))   # Pr(sigma g > k - 1/2)
    up_hi = 0.5 * erfc((kp + 0.5) / (sigma * SQRT2))   # Pr(sigma g > k + 1/2)
    pp = up_lo - up_hi
    pp[..., 0] = 1.0 - 2.0 * up_hi[..., 0]             # v = 0: |sigma g| < 1/2
    if lim is not None:
        pp[..., -1] = up_lo[..., -1]                   # v = K takes the whole tail
    k = np.arange(-K, K + 1, dtype=np.float64)
    p = np.concatenate([pp[..., :0:-1], pp], axis=-1)
    return k, p


def moments(sigma, lim: int | None = 7):
    """(m2, m4) of one quantised component."""
    k, p = level_probs(sigma, lim)
    m2 = (p * k ** 2).sum(axis=-1)
    m4 = (p * k ** 4).sum(axis=-1)
    return m2, m4


def delta_of_sigma(sigma, lim: int | None = 7):
    """Mean offset of SK~ from 1 for components of rms sigma before quantisation."""
    m2, m4 = moments(sigma, lim)
    return m4 / (2.0 * m2 * m2) - 1.5


def sigma_of_power(mu, lim: int = 7, lo: float = 1e-3, hi: float = 1e3, iters: int = 200):
    """sigma with 2 m2(sigma) = mu (bisection in log sigma), clamped to [lo, hi]."""
    mu = np.atleast_1d(np.asarray(mu, dtype=np.float64))
    a = np.full(mu.shape, math.log(lo))
    b = np.full(mu.shape, math.log(hi))
    for _ in range(iters):
        c = 0.5 * (a + b)
        m2, _ = moments(np.exp(c), lim)
        below = 2.0 * m2 < mu
        a = np.where(below, c, a)
        b = np.where(below, b, c)
    return np.exp(0.5 * (a + b))


def delta_of_power(mu, lim: int = 7):
    return delta_of_sigma(sigma_of_power(mu, lim), lim)


def offset_table(M: int, B: int = 4096, k: int = 6, lim: int = 7) -> np.ndarray:
    """e[b] = rint(delta(mu_b) * 2^32 * (n-1)/(n+1)), mu_b = (b + 1/2) * 128 / B.

    One entry per power bucket; summed over inputs it is the shift of the Q
    thresholds that moves the centre from 1 to 1 + Avg(delta_i).
    """
    mu = (np.arange(B, dtype=np.float64) + 0.5) * 128.0 / B
    d = delta_of_power(mu, lim)
    x = d * 4294967296.0 * float(M - 1) / float(M + 1)
    return np.array([int(round(v)) for v in x], dtype=np.int64)
