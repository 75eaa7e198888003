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
"""

from __future__ import annotations

import numpy as np

from . import power_sums, sk_spec, thresholds


def bucket(P: np.ndarray, M: int, B: int = 4096, k: int = 6) -> np.ndarray:
    b = (P.astype(np.uint64) * np.uint64(B)) // np.uint64((1 << k) * M * 128)
    return np.minimum(b, np.uint64(B - 1)).astype(np.int64)


def served_flags(frames: np.ndarray, M: int, N: int, e: np.ndarray, n_sigma: float = 3.0,
                 mean_offset: float = 0.0, k: int = 6, B: int = 4096, layout: int = 0,
                 P0: np.ndarray | None = None):
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
    for f in range(T):
        s1 = S1[f]
        if P is None:
            P = s1 << k
        valid = s1 > 0
        E[f] = int(e[bucket(P, M, B, k)][valid].sum())
        n = int(ne[f])
        m = (n == 0) or (Q[f] > t_hi[n] + E[f]) or (Q[f] < t_lo[n] + E[f])
        msk[f] = 1 if m else 0
        if not m:
            P = P - (P >> k) + s1
    return dict(Q=Q, neff=ne, sk=sk, mask=msk, E=E, P=P, S1=S1, S2=S2)
